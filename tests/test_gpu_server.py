"""Continuous-batching server (sw_server_*): requests joining while others run,
resident gauge fields, admission by memory budget, and each result bit-identical
alone and in the mix."""
import numpy as np
import pytest

import lattice_synth as ls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1312_3265_gb300 as m
    m.lib()
    return m


def pinned(shape):
    import torch
    return torch.zeros(shape, dtype=torch.complex128).pin_memory().numpy()


def links(dims, seed):
    import torch
    return torch.from_numpy(ls.su3_links(dims, seed, ls.PLAQ_EPS)).cuda()


ENGINES = [((4, 4, 4, 4), 0, 1), ((6, 4, 4, 6), 1, 1), ((4, 4, 2, 6), 0, 0), ((4, 4, 4, 4), 1, 2)]
# (dims, op, precision)


def make_server(sw, slots=3):
    srv = sw.Server(8 << 30)
    eng = []
    for k, (dims, op, prec) in enumerate(ENGINES):
        eng.append(srv.add_engine(dims, op, links(dims, 10 + k), 1.0, prec, slots))
    return srv, eng


def request(dims, op, seed):
    nc = 3 if op == 0 else 12
    chi = pinned((ls.volume(dims), nc))
    chi[:] = ls.gaussian_source(dims, nc, seed)
    return chi, pinned((ls.volume(dims), nc))


def test_result_alone_equals_result_in_mix(sw):
    # alone
    srv, eng = make_server(sw)
    probe = []
    for k, (dims, op, prec) in enumerate(ENGINES):
        chi, x = request(dims, op, 100 + k)
        rid = srv.submit(eng[k], chi, x, 0.05 + 0.01 * k, 1e-9)
        srv.drain(120)
        (got_id, info), = srv.poll()
        assert got_id == rid and info.status == sw.SW_OK and info.true_rel_resid <= 1e-9
        probe.append(x.copy())
    srv.close()
    # in a mix: 40 requests over the four engines (3 slots each), the probes in the middle
    srv, eng = make_server(sw)
    mix = {}
    rng = np.random.default_rng(0)
    ids = {}
    for j in range(40):
        k = int(rng.integers(0, 4))
        dims, op, prec = ENGINES[k]
        if j == 20:
            for kk, (d2, o2, p2) in enumerate(ENGINES):
                chi, x = request(d2, o2, 100 + kk)
                ids[srv.submit(eng[kk], chi, x, 0.05 + 0.01 * kk, 1e-9)] = ("probe", kk, x)
        chi, x = request(dims, op, 1000 + j)
        ids[srv.submit(eng[k], chi, x, float(rng.uniform(0.02, 0.2)), 1e-8)] = ("bg", k, x)
    srv.drain(300)
    done = dict(srv.poll(4096))
    assert set(done) == set(ids)
    for rid, (kind, k, x) in ids.items():
        assert done[rid].status == sw.SW_OK
        if kind == "probe":
            mix[k] = x
    srv.close()
    for k in range(4):
        assert np.array_equal(mix[k], probe[k]), f"engine {k}"


def test_server_matches_cgne_solve(sw):
    import torch
    dims, op = (6, 4, 4, 6), 1
    U = links(dims, 3)
    srv = sw.Server(4 << 30)
    e = srv.add_engine(dims, op, U, 1.0, sw.SW_PREC_F32_RELIABLE, 2)
    outs = []
    for j in range(5):  # more requests than slots: they queue and join as slots free up
        chi, x = request(dims, op, 50 + j)
        srv.submit(e, chi, x, 0.1, 1e-9)
        outs.append((chi, x))
    srv.drain(120)
    infos = srv.poll()
    assert len(infos) == 5 and all(i.status == sw.SW_OK for _, i in infos)
    srv.close()
    for chi, x in outs:
        cd = torch.from_numpy(chi.reshape(-1, 4, 3).copy()).cuda()
        xd = torch.zeros_like(cd)
        sw.cgne_solve(dims, op, U, None, cd, xd, 0.1, 1.0, 1e-9, 100000, sw.SW_PREC_F32_RELIABLE)
        assert np.array_equal(xd.cpu().numpy().reshape(x.shape), x)


def test_budget_and_arguments(sw):
    dims = (8, 8, 8, 8)
    U = links(dims, 1)
    srv = sw.Server(1 << 20)  # 1 MiB: no engine fits
    with pytest.raises(sw.SWError) as e:
        srv.add_engine(dims, 0, U, 1.0, sw.SW_PREC_F32_RELIABLE, 4)
    assert e.value.code == -6
    srv.close()
    srv = sw.Server(1 << 30)
    eng = srv.add_engine(dims, 0, U, 1.0, sw.SW_PREC_F32_RELIABLE, 4)
    chi, x = request(dims, 0, 1)
    with pytest.raises(sw.SWError):
        srv.submit(eng + 5, chi, x, 0.1)
    with pytest.raises(sw.SWError):
        srv.submit(eng, chi, x, 0.1, tol=2.0)
    with pytest.raises(sw.SWError):  # engines are fixed once serving has started
        srv.submit(eng, chi, x, 0.1)
        srv.add_engine(dims, 0, U, 1.0, sw.SW_PREC_F32_RELIABLE, 4)
    srv.drain(60)
    srv.close()
