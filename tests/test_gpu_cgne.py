"""GPU CGNE (Eq. 2) against the oracle, through the C ABI.

Bar: FP64 true relative residual |b - A x|/|b| <= tol (1e-8, recomputed by the
oracle's operator on the GPU's x), solution within 1e-6 relative of the
oracle's CG solution (solved to 1e-12), FP64 iteration counts within 2% (or 2
iterations) of the oracle's at the same tolerance.
"""
import numpy as np
import pytest

import lattice_synth as ls
from oracle import Lattice, operators as ops
from oracle.cg import cgne

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1312_3265_gb300 as m
    m.lib()
    return m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class Problem:
    def __init__(self, sw, dims, op, seed, eps, mass, apbc=False, r=1.0):
        import torch
        self.dims, self.op, self.mass, self.apbc, self.r = dims, op, mass, apbc, r
        self.lat = Lattice(dims, apbc)
        self.Uh = ls.su3_links(dims, seed, eps)
        self.U = dev(self.Uh)
        self.U4 = self.lat.links(self.Uh)
        self.nc = 3 if op == sw.SW_OP_STAGGERED_WILSON else 12
        self.internal = (3,) if self.nc == 3 else (4, 3)
        self.W = None
        if self.nc == 3:
            self.W = torch.empty((self.lat.volume, 8, 3, 3), dtype=torch.complex128, device="cuda")
            sw.sw_hypercube_build(dims, self.U, self.W)

    def D(self, v, dag=False):
        if self.nc == 3:
            return ops.sw_dslash(self.lat, self.U4, v, self.mass, self.r, dag)
        return ops.wilson_dslash(self.lat, self.U4, v, self.mass, self.r, dag)

    def field(self, flat):
        return self.lat.field(flat.reshape((-1,) + self.internal), self.internal)

    def oracle(self, chi_flat, tol):
        x, info = cgne(lambda v: self.D(v), lambda v: self.D(v, True), self.field(chi_flat), tol, 100000)
        return x.reshape(-1), info

    def true_resid(self, chi_flat, x_flat):
        b = self.D(self.field(chi_flat), True)
        r = b - self.D(self.D(self.field(x_flat)), True)
        return np.linalg.norm(r) / np.linalg.norm(b)

    def solve(self, sw, chi_flat, tol, prec, max_iter=100000, x0=None):
        import torch
        chi = dev(chi_flat.reshape((-1,) + self.internal))
        x = torch.zeros_like(chi) if x0 is None else dev(x0.reshape((-1,) + self.internal))
        info = sw.cgne_solve(self.dims, self.op, self.U, self.W, chi, x, self.mass, self.r, tol, max_iter, prec,
                             self.apbc)
        torch.cuda.synchronize()
        return x.cpu().numpy().reshape(-1), info


def check(sw, P, chi, prec, tol=1e-8):
    x, info = P.solve(sw, chi, tol, prec)
    assert info.status == sw.SW_OK
    assert info.true_rel_resid <= tol
    rr = P.true_resid(chi, x)
    assert rr <= tol * 1.01
    # the solver's own FP64 residual recomputation agrees with the oracle's
    assert abs(info.true_rel_resid - rr) <= 1e-13 + 1e-3 * rr
    ref, _ = P.oracle(chi, 1e-12)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6
    return x, info


def test_small_workload_sw(sw):
    """4^4 staggered Wilson: eps = 0.3 links from seed 0, r = 1, m = 0.05, point
    source at the origin, colour 0, tol 1e-8."""
    P = Problem(sw, (4, 4, 4, 4), sw.SW_OP_STAGGERED_WILSON, 0, ls.LINK_EPS_SMALL, 0.05)
    chi = ls.point_source(P.dims, 3, 0).reshape(-1)
    _, info = check(sw, P, chi, sw.SW_PREC_F64)
    _, oinfo = P.oracle(chi, 1e-8)
    assert abs(info.iters - oinfo["iters"]) <= max(2, 0.02 * oinfo["iters"])
    check(sw, P, chi, sw.SW_PREC_F32_RELIABLE)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("alpha", [0, 7])
def test_small_workload_wilson(sw, prec, alpha):
    P = Problem(sw, (4, 4, 4, 4), sw.SW_OP_WILSON, 0, ls.LINK_EPS_SMALL, 0.05)
    chi = ls.point_source(P.dims, 12, alpha).reshape(-1)
    _, info = check(sw, P, chi, prec)
    if prec == sw.SW_PREC_F64:
        _, oinfo = P.oracle(chi, 1e-8)
        assert abs(info.iters - oinfo["iters"]) <= max(2, 0.02 * oinfo["iters"])


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_ragged_antiperiodic(sw, op, prec):
    P = Problem(sw, (6, 6, 4, 6), op, 2, ls.PLAQ_EPS, 0.1, apbc=True)
    chi = ls.gaussian_source(P.dims, P.nc, 3).reshape(-1)
    check(sw, P, chi, prec)


def test_wilson_general_r(sw):
    P = Problem(sw, (4, 4, 2, 4), sw.SW_OP_WILSON, 5, 0.4, 0.1, r=0.75)
    chi = ls.gaussian_source(P.dims, 12, 1).reshape(-1)
    check(sw, P, chi, sw.SW_PREC_F64)
    check(sw, P, chi, sw.SW_PREC_F32_RELIABLE)
    check(sw, P, chi, sw.SW_PREC_F16_RELIABLE)


def test_edge_cases(sw):
    P = Problem(sw, (2, 2, 2, 2), sw.SW_OP_STAGGERED_WILSON, 1, 0.3, 0.1)
    # zero source: x = 0 exactly, even from a non-zero guess (FP64 and the
    # mixed modes, whose right-hand side comes from the inner-precision operator)
    zero = np.zeros(P.lat.volume * 3, dtype=np.complex128)
    for prec in (0, 1, 2):
        x, info = P.solve(sw, zero, 1e-8, prec, x0=np.ones_like(zero))
        assert info.status == sw.SW_OK and np.all(x == 0)
    # max_iter reached: status SW_NOT_CONVERGED, true residual reported
    P4 = Problem(sw, (4, 4, 4, 4), sw.SW_OP_WILSON, 0, 0.3, 0.01)
    chi = ls.point_source(P4.dims, 12, 0).reshape(-1)
    x, info = P4.solve(sw, chi, 1e-10, 0, max_iter=3)
    assert info.status == sw.SW_NOT_CONVERGED and info.iters == 3
    assert abs(info.true_rel_resid - P4.true_resid(chi, x)) < 1e-6
    # the guess is used: starting from the solution needs no iteration (the
    # FP64 residual of the guess decides, in every precision mode)
    xs, _ = P4.solve(sw, chi, 1e-9, 0)
    for prec in (0, 1, 2):
        _, info = P4.solve(sw, chi, 1e-8, prec, x0=xs)
        assert info.status == sw.SW_OK and info.iters == 0 and info.true_rel_resid <= 1e-8
    # a NaN source is reported, not iterated on
    bad = chi.copy()
    bad[5] = np.nan
    with pytest.raises(sw.SWError) as e:
        P4.solve(sw, bad, 1e-8, 1)
    assert e.value.code == -5
    # free field on 2^4: CG ends in at most 2 iterations (2 distinct eigenvalues)
    F = Problem(sw, (2, 2, 2, 2), sw.SW_OP_STAGGERED_WILSON, 1, 0.0, 0.1)
    chi = ls.gaussian_source(F.dims, 3, 4).reshape(-1)
    _, info = F.solve(sw, chi, 1e-12, 0)
    assert info.status == sw.SW_OK and info.iters <= 2


def test_full_size_solve(sw):
    """16^3x32, mean plaquette 0.59 links: mixed-precision solves of both operators
    meet the FP64 true residual checked by the oracle's operator."""
    for op in (sw.SW_OP_STAGGERED_WILSON, sw.SW_OP_WILSON):
        P = Problem(sw, (16, 16, 16, 32), op, 0, ls.PLAQ_EPS, 0.1)
        chi = ls.point_source(P.dims, P.nc, 0).reshape(-1)
        for prec in (sw.SW_PREC_F32_RELIABLE, sw.SW_PREC_F16_RELIABLE):
            x, info = P.solve(sw, chi, 1e-8, prec)
            assert info.status == sw.SW_OK and info.true_rel_resid <= 1e-8
            assert P.true_resid(chi, x) <= 1.01e-8


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_is_bitwise_single(sw, op, prec):
    """Each system of a batch gives bit-identical results to solving it alone:
    the per-system arithmetic and the reduction order (fixed 128-site tiles) do
    not depend on the batch.  5 systems (not a multiple of the register-blocking
    width), different masses and sources."""
    import torch
    P = Problem(sw, (6, 4, 4, 6), op, 7, ls.PLAQ_EPS, 0.1, apbc=True)
    masses = [0.05, 0.1, 0.2, 0.07, 0.3]
    chis = np.stack([ls.gaussian_source(P.dims, P.nc, 20 + i).reshape((-1,) + P.internal) for i in range(5)])
    chi = dev(chis)
    x = torch.zeros_like(chi)
    rc, infos = sw.cgne_solve_batch(P.dims, op, P.U, P.W, chi, x, masses, 1.0, 1e-9, 10000, prec, True)
    assert rc == sw.SW_OK
    xb = x.cpu().numpy()
    for i, m in enumerate(masses):
        xi = torch.zeros_like(chi[i])
        info = sw.cgne_solve(P.dims, op, P.U, P.W, chi[i].contiguous(), xi, m, 1.0, 1e-9, 10000, prec, True)
        assert info.iters == infos[i].iters and info.reliable_updates == infos[i].reliable_updates
        assert np.array_equal(xi.cpu().numpy(), xb[i])
        assert infos[i].true_rel_resid <= 1e-9


def test_reliable_update_delta_param(sw):
    P = Problem(sw, (6, 6, 4, 6), sw.SW_OP_WILSON, 2, ls.PLAQ_EPS, 0.05)
    chi = ls.gaussian_source(P.dims, 12, 3).reshape(-1)
    old = sw.sw_get_param(sw.SW_PARAM_RELIABLE_DELTA)
    try:
        counts = {}
        for d in (0.1, 1e-3):
            sw.sw_set_param(sw.SW_PARAM_RELIABLE_DELTA, d)
            x, info = P.solve(sw, chi, 1e-9, sw.SW_PREC_F32_RELIABLE)
            assert info.status == sw.SW_OK and P.true_resid(chi, x) <= 1.01e-9
            counts[d] = info.reliable_updates
        assert counts[1e-3] < counts[0.1]
        with pytest.raises(sw.SWError):
            sw.sw_set_param(sw.SW_PARAM_RELIABLE_DELTA, 1.5)
    finally:
        sw.sw_set_param(sw.SW_PARAM_RELIABLE_DELTA, old)


def test_condition_number_estimates(sw):
    """Ritz values from CG's coefficients against the paper's condition number
    kappa = lmax/lmin of (D+m)^+(D+m) (Sec. 3): the free-field closed forms on 4^4
    (SW: lmax = 4 + (1+m)^2, lmin = m^2; Wilson: (8+m)^2 and m^2), and the dense
    oracle spectrum on an interacting 4^4 field."""
    from oracle import dense
    m = 0.1
    for op, lmax in ((sw.SW_OP_STAGGERED_WILSON, 4 + (1 + m) ** 2), (sw.SW_OP_WILSON, (8 + m) ** 2)):
        P = Problem(sw, (4, 4, 4, 4), op, 1, 0.0, m)
        chi = ls.gaussian_source(P.dims, P.nc, 5).reshape(-1)
        _, info = P.solve(sw, chi, 1e-12, sw.SW_PREC_F64)
        assert abs(info.lambda_max - lmax) < 1e-6 * lmax
        assert abs(info.lambda_min - m * m) < 1e-6 * m * m
    P = Problem(sw, (4, 4, 4, 4), sw.SW_OP_STAGGERED_WILSON, 0, ls.LINK_EPS_SMALL, 0.05)
    ev = dense.normal_spectrum(dense.sw_matrix(P.lat, P.U4, 0.05))
    chi = ls.gaussian_source(P.dims, 3, 6).reshape(-1)
    for prec in (sw.SW_PREC_F64, sw.SW_PREC_F32_RELIABLE):
        _, info = P.solve(sw, chi, 1e-12, prec)
        assert abs(info.lambda_max / ev[-1] - 1) < 1e-3
        # Ritz values approach lambda_min from above and converge last when the
        # low end of the spectrum is clustered: 1% after a 1e-12 solve
        assert ev[0] * (1 - 1e-9) <= info.lambda_min < ev[0] * 1.01


@pytest.mark.parametrize("op,widths", [(0, (1, 2, 4)), (1, (1, 2, 4))])
def test_register_blocking_widths(sw, op, widths):
    """The FP32 stencils computing 1, 2 or 4 systems per thread solve the same
    systems to the same FP64 residual (7 systems: ragged groups)."""
    import torch
    P = Problem(sw, (6, 4, 4, 6), op, 8, ls.PLAQ_EPS, 0.1)
    masses = [0.05, 0.1, 0.2, 0.07, 0.3, 0.02, 0.15]
    chis = np.stack([ls.gaussian_source(P.dims, P.nc, 40 + i).reshape((-1,) + P.internal) for i in range(7)])
    chi = dev(chis)
    key = sw.SW_PARAM_NS_SW if op == 0 else sw.SW_PARAM_NS_WILSON
    old = sw.sw_get_param(key)
    try:
        for ns in widths:
            sw.sw_set_param(key, ns)
            x = torch.zeros_like(chi)
            rc, infos = sw.cgne_solve_batch(P.dims, op, P.U, P.W, chi, x, masses, 1.0, 1e-9, 10000,
                                            sw.SW_PREC_F32_RELIABLE)
            assert rc == sw.SW_OK
            xs = x.cpu().numpy()
            for i, m in enumerate(masses):
                P.mass = m
                assert P.true_resid(chis[i].reshape(-1), xs[i].reshape(-1)) <= 1.01e-9
    finally:
        sw.sw_set_param(key, old)



def test_half_precision_needs_su3_links(sw):
    """FP16 storage keeps two rows of each link and rebuilds the third, so links
    that are not SU(3) are refused before anything runs."""
    import torch
    P = Problem(sw, (4, 4, 4, 4), sw.SW_OP_WILSON, 3, 0.3, 0.1)
    chi = dev(ls.gaussian_source(P.dims, 12, 2).reshape(-1, 4, 3))
    x = torch.zeros_like(chi)
    with pytest.raises(sw.SWError) as e:
        sw.cgne_solve(P.dims, P.op, P.U * 1.01, None, chi, x, 0.1, 1.0, 1e-8, 1000, sw.SW_PREC_F16_RELIABLE)
    assert e.value.code == -8
    info = sw.cgne_solve(P.dims, P.op, P.U * 1.01, None, chi, x, 0.1, 1.0, 1e-8, 1000, sw.SW_PREC_F32_RELIABLE)
    assert info.status == sw.SW_OK  # FP32 keeps all 18 reals: any links work


def test_graph_replay_is_bitwise_launches(sw):
    """Chunks of iterations replayed as a captured CUDA graph, with the FP64
    reliable updates of some systems running on a side stream while the others
    iterate, give exactly the results of launching the kernels one by one on
    one stream (three masses: the systems reach their updates in different
    rounds)."""
    import torch
    P = Problem(sw, (6, 4, 4, 6), sw.SW_OP_WILSON, 9, ls.PLAQ_EPS, 0.05)
    chis = np.stack([ls.gaussian_source(P.dims, 12, 60 + i).reshape(-1, 4, 3) for i in range(3)])
    chi = dev(chis)
    out = {}
    old = sw.sw_get_param(sw.SW_PARAM_GRAPHS)
    try:
        for gflag in (0, 1):
            sw.sw_set_param(sw.SW_PARAM_GRAPHS, gflag)
            x = torch.zeros_like(chi)
            rc, infos = sw.cgne_solve_batch(P.dims, P.op, P.U, None, chi, x, [0.05, 0.1, 0.2], 1.0, 1e-10, 10000,
                                            sw.SW_PREC_F32_RELIABLE)
            assert rc == sw.SW_OK and infos[0].iters > 3 * 16  # several chunks, so replays happen
            out[gflag] = x.cpu().numpy()
    finally:
        sw.sw_set_param(sw.SW_PARAM_GRAPHS, old)
    assert np.array_equal(out[0], out[1])


def test_autotune_picks_a_width_and_solves(sw):
    import torch
    P = Problem(sw, (8, 8, 8, 8), sw.SW_OP_STAGGERED_WILSON, 4, ls.PLAQ_EPS, 0.1)
    old = sw.sw_get_param(sw.SW_PARAM_NS_SW)
    try:
        best, times = sw.sw_autotune(P.dims, P.op, P.U, P.W, 6, sw.SW_PREC_F32_RELIABLE, iters=32)
        assert best in (1, 2, 4) and sw.sw_get_param(sw.SW_PARAM_NS_SW) == best
        assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
        chi = ls.gaussian_source(P.dims, 3, 8).reshape(-1)
        check(sw, P, chi, sw.SW_PREC_F32_RELIABLE)
    finally:
        sw.sw_set_param(sw.SW_PARAM_NS_SW, old)


@pytest.mark.parametrize("op", ["sw", "wilson"])
def test_autotune_layout_picks_width_and_site_order(sw, op):
    """The width x site-order autotuner times every pair (3 widths x the
    lexicographic order and the site-block shapes), sets the fastest, and the
    solver then converges with that layout."""
    P = (Problem(sw, (8, 8, 8, 8), sw.SW_OP_STAGGERED_WILSON, 4, ls.PLAQ_EPS, 0.1) if op == "sw"
         else Problem(sw, (8, 8, 8, 8), sw.SW_OP_WILSON, 4, ls.PLAQ_EPS, 0.1))
    key = sw.SW_PARAM_NS_SW if op == "sw" else sw.SW_PARAM_NS_WILSON
    old = (sw.sw_get_param(key), sw.sw_get_param(sw.SW_PARAM_SITE_BLOCKING))
    try:
        best, times = sw.sw_autotune_layout(P.dims, P.op, P.U, P.W, 5, sw.SW_PREC_F32_RELIABLE, iters=24)
        assert set(times) == {(w, b) for w in (1, 2, 4) for b in range(sw.SW_SITE_SHAPES)}
        assert best in times and times[best] == min(times.values()) and all(t > 0 for t in times.values())
        assert (sw.sw_get_param(key), sw.sw_get_param(sw.SW_PARAM_SITE_BLOCKING)) == best
        nc = 3 if op == "sw" else 12
        chi = ls.gaussian_source(P.dims, nc, 9).reshape(-1)
        check(sw, P, chi, sw.SW_PREC_F32_RELIABLE)
    finally:
        sw.sw_set_param(key, old[0])
        sw.sw_set_param(sw.SW_PARAM_SITE_BLOCKING, old[1])


@pytest.mark.parametrize("blocking", range(6))
@pytest.mark.parametrize("gfast", [0, 1])
def test_site_order_and_grid_order(sw, blocking, gfast):
    """The packed fields' site order (lexicographic or any site-block shape)
    and the stencil grid order solve the same systems; the grid order does not
    even change a bit (the reductions go over the same site tiles)."""
    import torch
    P = Problem(sw, (8, 4, 6, 8), sw.SW_OP_STAGGERED_WILSON, 6, ls.PLAQ_EPS, 0.07, apbc=True)
    chis = np.stack([ls.gaussian_source(P.dims, 3, 70 + i) for i in range(5)])
    chi = dev(chis)
    old = (sw.sw_get_param(sw.SW_PARAM_SITE_BLOCKING), sw.sw_get_param(sw.SW_PARAM_GROUP_FAST))
    outs = {}
    try:
        sw.sw_set_param(sw.SW_PARAM_SITE_BLOCKING, blocking)
        for gf in (gfast, 1 - gfast):
            sw.sw_set_param(sw.SW_PARAM_GROUP_FAST, gf)
            for prec in (sw.SW_PREC_F32_RELIABLE, sw.SW_PREC_F16_RELIABLE):
                x = torch.zeros_like(chi)
                rc, infos = sw.cgne_solve_batch(P.dims, P.op, P.U, P.W, chi, x, [0.07] * 5, 1.0, 1e-9, 10000, prec,
                                                True)
                assert rc == sw.SW_OK
                outs[(gf, prec)] = x.cpu().numpy()
                for i in range(5):
                    assert P.true_resid(chis[i].reshape(-1), outs[(gf, prec)][i].reshape(-1)) <= 1.01e-9
    finally:
        sw.sw_set_param(sw.SW_PARAM_SITE_BLOCKING, old[0])
        sw.sw_set_param(sw.SW_PARAM_GROUP_FAST, old[1])
    for prec in (sw.SW_PREC_F32_RELIABLE, sw.SW_PREC_F16_RELIABLE):
        assert np.array_equal(outs[(0, prec)], outs[(1, prec)])


def test_concurrent_solves_from_two_threads(sw):
    """Two host threads solving a staggered Wilson and a Wilson batch at the same
    time, each on its own stream, get bit-identical results to solving them one
    after the other (the entry points are thread-safe; every solve owns its
    workspace, status buffers and side stream)."""
    import threading
    import torch
    dims = (6, 4, 4, 6)
    Ps = Problem(sw, dims, sw.SW_OP_STAGGERED_WILSON, 11, ls.PLAQ_EPS, 0.1, apbc=True)
    Pw = Problem(sw, dims, sw.SW_OP_WILSON, 11, ls.PLAQ_EPS, 0.1, apbc=True)
    ms, mw = [0.05, 0.1, 0.2], [0.05, 0.1, 0.2, 0.07]
    chs = dev(np.stack([ls.gaussian_source(dims, 3, 80 + i).reshape(-1, 3) for i in range(3)]))
    chw = dev(np.stack([ls.gaussian_source(dims, 12, 90 + i).reshape(-1, 4, 3) for i in range(4)]))

    def run(P, ch, masses, stream):
        with torch.cuda.stream(stream):
            x = torch.zeros_like(ch)
            rc, infos = sw.cgne_solve_batch(dims, P.op, P.U, P.W, ch, x, masses, 1.0, 1e-9, 10000,
                                            sw.SW_PREC_F32_RELIABLE, True, stream=stream)
        stream.synchronize()
        return rc, infos, x.cpu().numpy()

    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ref_s, ref_w = run(Ps, chs, ms, s1), run(Pw, chw, mw, s2)
    out = {}
    th = threading.Thread(target=lambda: out.__setitem__("s", run(Ps, chs, ms, s1)))
    th.start()
    out["w"] = run(Pw, chw, mw, s2)
    th.join()
    for ref, got in ((ref_s, out["s"]), (ref_w, out["w"])):
        assert ref[0] == sw.SW_OK and got[0] == sw.SW_OK
        assert [i.iters for i in ref[1]] == [i.iters for i in got[1]]
        assert np.array_equal(ref[2], got[2])


def test_solve_beside_bulk_copies_on_another_stream(sw):
    """A batch solved while another stream keeps the copy engines busy with
    bulk host<->device copies gives bit-identical results and iteration counts
    to the same batch solved alone (the solver's status words move by kernel
    through mapped pinned memory, beside those copies)."""
    import torch
    dims = (6, 4, 4, 6)
    P = Problem(sw, dims, sw.SW_OP_WILSON, 12, ls.PLAQ_EPS, 0.1, apbc=True)
    masses = [0.05, 0.1, 0.2]
    ch = dev(np.stack([ls.gaussian_source(dims, 12, 100 + i).reshape(-1, 4, 3) for i in range(3)]))

    def run():
        x = torch.zeros_like(ch)
        rc, infos = sw.cgne_solve_batch(dims, P.op, P.U, None, ch, x, masses, 1.0, 1e-9, 10000,
                                        sw.SW_PREC_F32_RELIABLE, True)
        torch.cuda.synchronize()
        return rc, [i.iters for i in infos], x.cpu().numpy()

    ref = run()
    n = 64 << 20  # 256 MB each way
    h_up = torch.ones(n, dtype=torch.float32).pin_memory()
    h_dn = torch.empty(n, dtype=torch.float32).pin_memory()
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    cs = torch.cuda.Stream()
    with torch.cuda.stream(cs):
        for _ in range(4):
            d.copy_(h_up, non_blocking=True)
            h_dn.copy_(d, non_blocking=True)
    got = run()
    cs.synchronize()
    assert ref[0] == sw.SW_OK and got[0] == sw.SW_OK
    assert ref[1] == got[1]
    assert np.array_equal(ref[2], got[2])
    assert float(h_dn[::1 << 20].min()) == 1.0


def test_workspace_pool_keeps_and_trims(sw):
    """A solve's device workspace comes from the library's pool: it stays
    reserved after the solve (for the next call), sw_trim_workspace hands the
    unused part back, and a solve after the trim allocates again and gives a
    bit-identical result."""
    dims = (6, 4, 4, 6)
    P = Problem(sw, dims, sw.SW_OP_WILSON, 13, ls.PLAQ_EPS, 0.1, apbc=True)
    chi = ls.gaussian_source(dims, 12, 5).reshape(-1)
    out = []
    for _ in range(2):
        x, info = P.solve(sw, chi, 1e-9, sw.SW_PREC_F32_RELIABLE)
        assert info.status == sw.SW_OK
        held = sw.sw_workspace_reserved()
        assert held > 0
        sw.sw_trim_workspace()
        assert sw.sw_workspace_reserved() < held
        out.append(x)
    assert np.array_equal(out[0], out[1])


def test_bench_batch_at_full_size(sw):
    """The bench's launch configuration at its full size: one 16^3x32
    configuration (mean plaquette 0.59), 12 staggered Wilson systems (3 colour
    point sources x 4 masses) and 48 Wilson systems (12 spin-colour point
    sources x 4 masses), mass-major, each operator in one cgne_solve_batch with
    the library's defaults (FP32 inner iterations, CUDA graphs, reliable
    updates beside the iterations, register blocking).  Every system meets the
    FP64 true residual 1e-8, computed with the FP64 operators (which
    test_gpu_dslash pins to the oracle site by site at full size), and at
    sampled sites the oracle's one-site operator reproduces (D+m) x of the
    first and last system of each batch."""
    import torch
    from oracle import site
    dims, masses, tol = (16, 16, 16, 32), (0.02, 0.05, 0.1, 0.2), 1e-8
    V = ls.volume(dims)
    Uh = ls.su3_links(dims, 0, ls.PLAQ_EPS, processes=8)
    U = dev(Uh)
    W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
    sw.sw_hypercube_build(dims, U, W)
    rng = np.random.default_rng(11)
    sites = [0, 1, V - 1, 16 * 16 * 16 - 1] + [int(v) for v in rng.integers(0, V, 6)]
    for op, nsrc, shape in ((sw.SW_OP_STAGGERED_WILSON, 3, (V, 3)), (sw.SW_OP_WILSON, 12, (V, 4, 3))):
        chis = np.stack([ls.point_source(dims, 3 if nsrc == 3 else 12, a).reshape(shape)
                         for m in masses for a in range(nsrc)])
        ms = [m for m in masses for _ in range(nsrc)]
        chi = dev(chis)
        x = torch.zeros_like(chi)
        rc, infos = sw.cgne_solve_batch(dims, op, U, W if op == sw.SW_OP_STAGGERED_WILSON else None, chi, x, ms,
                                        1.0, tol, 100000, sw.SW_PREC_F32_RELIABLE)
        assert rc == sw.SW_OK and all(i.status == sw.SW_OK and i.true_rel_resid <= tol for i in infos)

        def apply(v, m, dag):
            out = torch.empty_like(v)
            if op == sw.SW_OP_STAGGERED_WILSON:
                sw.sw_dslash_apply(dims, U, W, v, out, m, 1.0, dag)
            else:
                sw.wilson_dslash_apply(dims, U, v, out, m, 1.0, dag)
            return out

        for k, m in enumerate(ms):
            Dx = apply(x[k], m, False)
            b = apply(chi[k], m, True)
            r = b - apply(Dx, m, True)
            rel = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b))
            assert rel <= 1.01 * tol, (op, k, rel)
            if k in (0, len(ms) - 1):
                xh, got = x[k].cpu().numpy(), Dx.cpu().numpy()
                # (D+m)x is ~chi, i.e. ~0 away from the source: a cancellation
                # of O(|x|) terms, so the rounding scale is |x|, not the output
                scale = np.abs(xh).max()
                for n in sites:
                    if op == sw.SW_OP_STAGGERED_WILSON:
                        want = site.sw_dslash_site(Uh, xh, dims, n, m, 1.0, False, False)
                    else:
                        want = site.wilson_dslash_site(Uh, xh, dims, n, m, 1.0, False, False)
                    assert np.abs(got[n] - want).max() <= 1e-12 * scale, (op, k, n)
        del chi, x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("op,prec", [(1, 1), (0, 1), (1, 2), (0, 0)])
def test_persistent_graph_is_bitwise_host_rounds(sw, op, prec):
    """The whole solve as one CUDA graph (admission, a conditional WHILE node
    over rounds of reliable updates beside chunks of iterations, the status
    read) gives bit for bit the solutions and iteration counts of the
    host-driven rounds, and issues fewer host-visible launches; three masses,
    so the systems take their reliable updates in different rounds."""
    import torch
    P = Problem(sw, (6, 4, 4, 6), op, 14, ls.PLAQ_EPS, 0.05, apbc=True)
    masses = [0.05, 0.1, 0.2]
    chis = np.stack([ls.gaussian_source(P.dims, P.nc, 110 + i).reshape((-1,) + P.internal) for i in range(3)])
    chi = dev(chis)
    out, iters = {}, {}
    old = sw.sw_get_param(sw.SW_PARAM_PERSISTENT)
    try:
        for pflag in (0, 1):
            sw.sw_set_param(sw.SW_PARAM_PERSISTENT, pflag)
            x = torch.zeros_like(chi)
            rc, infos = sw.cgne_solve_batch(P.dims, P.op, P.U, P.W, chi, x, masses, 1.0, 1e-10, 10000, prec, True)
            assert rc == sw.SW_OK and all(i.true_rel_resid <= 1e-10 for i in infos)
            out[pflag] = x.cpu().numpy()
            iters[pflag] = [(i.iters, i.reliable_updates) for i in infos]
    finally:
        sw.sw_set_param(sw.SW_PARAM_PERSISTENT, old)
    assert iters[0] == iters[1]
    assert np.array_equal(out[0], out[1])
    for i, m in enumerate(masses):
        P.mass = m
        assert P.true_resid(chis[i].reshape(-1), out[1][i].reshape(-1)) <= 1.01e-10


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", ["r1", "r075"])
def test_even_odd_wilson_matches_the_oracle(sw, prec, case):
    """Wilson CGNE on the even-odd Schur complement (SW_OP_WILSON_EVEN_ODD):
    the same solution as the oracle's unpreconditioned CG (1e-6 relative), the
    full system's FP64 true residual <= tol checked by the oracle's operator
    (and reported as the oracle computes it), fewer CG iterations than the
    unpreconditioned solve of the same system, initial guesses (exact: no
    iteration; perturbed: converges again); a batch of three masses gives each
    system's result bit for bit as alone."""
    import torch
    if case == "r1":
        P = Problem(sw, (6, 4, 4, 6), sw.SW_OP_WILSON, 16, ls.PLAQ_EPS, 0.1, apbc=True)
    else:
        P = Problem(sw, (4, 4, 2, 4), sw.SW_OP_WILSON, 5, 0.4, 0.1, r=0.75)
    chi = ls.gaussian_source(P.dims, 12, 140).reshape(-1)
    ref, _ = P.oracle(chi, 1e-12)
    x_un, info_un = P.solve(sw, chi, 1e-9, prec)
    P.op = sw.SW_OP_WILSON_EVEN_ODD
    x, info = P.solve(sw, chi, 1e-9, prec)
    assert info.status == sw.SW_OK and info.true_rel_resid <= 1e-9
    assert P.true_resid(chi, x) <= 1.01e-9
    assert abs(info.true_rel_resid - P.true_resid(chi, x)) <= 1e-13 + 1e-3 * info.true_rel_resid
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6
    assert info.iters < info_un.iters, (info.iters, info_un.iters)
    # an initial guess: the oracle's solution stops at admission; a perturbed
    # one converges again to the full system's tolerance
    x0, info0 = P.solve(sw, chi, 1e-9, prec, x0=ref)
    assert info0.status == sw.SW_OK and info0.iters == 0 and P.true_resid(chi, x0) <= 1.01e-9
    noise = 1e-3 * np.linalg.norm(ref) / np.sqrt(ref.size) * ls.gaussian_source(P.dims, 12, 141).reshape(-1)
    x1, info1 = P.solve(sw, chi, 1e-9, prec, x0=ref + noise)
    assert info1.status == sw.SW_OK and 0 < info1.iters and P.true_resid(chi, x1) <= 1.01e-9
    assert abs(info1.true_rel_resid - P.true_resid(chi, x1)) <= 1e-13 + 1e-3 * info1.true_rel_resid
    # batch of three masses = each alone
    masses = [0.05, 0.1, 0.2]
    chis = np.stack([ls.gaussian_source(P.dims, 12, 150 + i).reshape(-1, 4, 3) for i in range(3)])
    chd = dev(chis)
    xb = torch.zeros_like(chd)
    rc, infos = sw.cgne_solve_batch(P.dims, P.op, P.U, None, chd, xb, masses, P.r, 1e-9, 10000, prec, P.apbc)
    assert rc == sw.SW_OK
    for i, m in enumerate(masses):
        xi = torch.zeros_like(chd[i])
        inf = sw.cgne_solve(P.dims, P.op, P.U, None, chd[i].contiguous(), xi, m, P.r, 1e-9, 10000, prec, P.apbc)
        assert inf.iters == infos[i].iters
        assert np.array_equal(xi.cpu().numpy(), xb[i].cpu().numpy())
        P.mass = m
        assert P.true_resid(chis[i].reshape(-1), xb[i].cpu().numpy().reshape(-1)) <= 1.01e-9


def test_wilson_lean_form_is_bitwise_default_form(sw):
    """The two forms of the spin-projected FP32 Wilson stencil
    (SW_PARAM_WILSON_LEAN: the lean one at 8 blocks per SM, the default one at
    7) perform the same operations in the same order: a mixed-precision batch
    (ragged masses, antiperiodic) and the inner operator itself, both ways,
    give bit-identical results."""
    import torch
    P = Problem(sw, (6, 4, 4, 6), sw.SW_OP_WILSON, 23, ls.PLAQ_EPS, 0.1, apbc=True)
    masses = [0.05, 0.1, 0.2, 0.07, 0.3]
    chis = np.stack([ls.gaussian_source(P.dims, 12, 60 + i).reshape(-1, 4, 3) for i in range(5)])
    chi = dev(chis)
    old = sw.sw_get_param(sw.SW_PARAM_WILSON_LEAN)
    out = {}
    try:
        for form in (1, 0):
            sw.sw_set_param(sw.SW_PARAM_WILSON_LEAN, form)
            x = torch.zeros_like(chi)
            rc, infos = sw.cgne_solve_batch(P.dims, P.op, P.U, None, chi, x, masses, 1.0, 1e-9, 10000,
                                            sw.SW_PREC_F32_RELIABLE, True)
            assert rc == sw.SW_OK
            y = torch.zeros_like(chi)
            for dag in (False, True):
                sw.dslash_apply_inner(P.dims, P.op, P.U, None, chi, y, masses, 1.0, dag, sw.SW_PREC_F32_RELIABLE, True)
                out[(form, dag)] = y.cpu().numpy()
            out[form] = (x.cpu().numpy(), [(i.iters, i.reliable_updates) for i in infos])
    finally:
        sw.sw_set_param(sw.SW_PARAM_WILSON_LEAN, old)
    assert out[1][1] == out[0][1]
    assert np.array_equal(out[1][0], out[0][0])
    for dag in (False, True):
        assert np.array_equal(out[(1, dag)], out[(0, dag)])
