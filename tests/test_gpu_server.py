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


ENGINES = [((4, 4, 4, 4), 0, 1), ((6, 4, 4, 6), 1, 1), ((4, 4, 2, 6), 0, 0), ((4, 4, 4, 4), 1, 2),
           ((6, 4, 4, 6), 0, 2)]
# (dims, op, precision): FP32, FP64 and FP16-storage engines of both operators


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
    # in a mix: 40 requests over the engines (3 slots each), the probes in the middle
    srv, eng = make_server(sw)
    mix = {}
    rng = np.random.default_rng(0)
    ids = {}
    for j in range(40):
        k = int(rng.integers(0, len(ENGINES)))
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
    for k in range(len(ENGINES)):
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


def field_request_bytes(sw, dims, U, op, prec, slots):
    """Device bytes the server charges for the engine of one (field, op,
    precision): measured by serving one request alone."""
    srv = sw.Server(8 << 30)
    f = srv.add_field(dims, U, slots)
    base = srv.stats()["bytes_charged"]
    chi, x = request(dims, op, 7)
    srv.submit_field(f, op, chi, x, 0.1, prec, tol=1e-9)
    srv.drain(120)
    st = srv.stats()
    srv.close()
    return base, st["bytes_charged"] - base


def test_field_requests_wait_for_memory(sw):
    """Admission by device memory: with a budget that holds the field and one
    engine but not two, a request for a second (operator, precision) on the
    same field waits until the first engine is idle and retired, then gets
    its own engine; each result is bit-identical to the same request served
    alone, and FP16 and FP32 engines alternate in the same budget."""
    dims = (6, 4, 4, 6)
    U = links(dims, 21)
    classes = [(1, sw.SW_PREC_F32_RELIABLE), (0, sw.SW_PREC_F16_RELIABLE), (1, sw.SW_PREC_F16_RELIABLE)]
    sizes = [field_request_bytes(sw, dims, U, op, prec, 2) for op, prec in classes]
    field_bytes = sizes[0][0]
    budget = field_bytes + max(b for _, b in sizes) + 1024
    assert budget < field_bytes + sizes[0][1] + sizes[1][1]
    # alone
    alone = []
    for k, (op, prec) in enumerate(classes):
        srv = sw.Server(8 << 30)
        f = srv.add_field(dims, U, 2)
        chi, x = request(dims, op, 300 + k)
        srv.submit_field(f, op, chi, x, 0.05 + 0.02 * k, prec, tol=1e-9)
        srv.drain(120)
        (_, info), = srv.poll()
        assert info.status == sw.SW_OK
        alone.append(x.copy())
        srv.close()
    # all three at once under the tight budget: they must take turns
    srv = sw.Server(budget)
    f = srv.add_field(dims, U, 2)
    ids = {}
    for k, (op, prec) in enumerate(classes):
        chi, x = request(dims, op, 300 + k)
        ids[srv.submit_field(f, op, chi, x, 0.05 + 0.02 * k, prec, tol=1e-9)] = (k, x)
    srv.drain(300)
    done = dict(srv.poll())
    st = srv.stats()
    srv.close()
    assert set(done) == set(ids) and all(i.status == sw.SW_OK for i in done.values())
    assert st["engines_created"] == 3 and st["engines_retired"] >= 2 and st["requests_waited_for_memory"] >= 1
    assert st["bytes_charged"] <= budget
    for rid, (k, x) in ids.items():
        assert np.array_equal(x, alone[k]), k


def test_field_request_that_can_never_fit_is_refused(sw):
    dims = (8, 8, 8, 8)
    U = links(dims, 2)
    srv = sw.Server(((8 ** 4) * 576) + (64 << 10))  # the field fits, no engine does
    f = srv.add_field(dims, U, 4)
    chi, x = request(dims, 1, 1)
    with pytest.raises(sw.SWError) as e:
        srv.submit_field(f, 1, chi, x, 0.1, sw.SW_PREC_F32_RELIABLE)
    assert e.value.code == -6
    srv.close()
