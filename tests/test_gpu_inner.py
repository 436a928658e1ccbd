"""The inner-precision operators of the mixed modes against the FP64 oracle,
element by element, through the C ABI (dslash_apply_inner runs the CG
iteration kernels themselves: cg_k1 for (D+m), cg_k2 for (D+m)^+).

These are the stencils that run every inner iteration; a wrong sign or a
dropped term there would otherwise only show up as more iterations, since the
FP64 reliable updates correct the solution.

Tolerance (worst-case rounding bounds, derived from the storage formats; the
per-component error is bounded by c * M with M = max over sites of the input's
2-norm per site and |out|max the largest output component):
  FP32 storage (u = 2^-24): input and link rounding perturb each 3x3 product
    component by at most 2 sqrt(6) u |psi(y)|; the FMA chains of one output
    component accumulate at most ~100 products (staggered Wilson: 8 hops and
    16 corners of 3 terms; Wilson: 8 projected hops of 6), so
    c32 = 100 u * (sum of the hop coefficients' norms, <= 9 + 4r + m) < 1e-4.
  FP16 storage (u = 2^-12 for the half-ulp of FP16 values in [0.5, 1) relative
    to the per-site scale; links and transports are stored the same way):
    c16 = 2 * 2 sqrt(6) u * (sum of hop norms) + output rounding sqrt(2) u |out|max.
A dropped hypercube corner costs r/16 |W psi| ~ 0.06 M, a wrong hop sign about
M: both far above either bound.
"""
import numpy as np
import pytest

import lattice_synth as ls
from oracle import Lattice, operators as ops

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U16 = 2.0 ** -12


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


def hop_norm_sum(nc, r, m):
    # staggered Wilson: 8 hops of 1/2, 16 corners of r/16, self r + m;
    # Wilson: 8 hops through the projectors (r -+ g)/2 (norm <= (r+1)/2), self 4r + m
    return 4.0 + r + r + abs(m) if nc == 3 else 4.0 * (r + 1.0) + 4.0 * r + abs(m)


def bound(nc, prec, r, m, M, outmax):
    s = hop_norm_sum(nc, r, m)
    if prec == 1:
        return 100.0 * U32 * s * M
    return 2.0 * 2.0 * np.sqrt(6.0) * U16 * s * M + np.sqrt(2.0) * U16 * outmax + 100.0 * U32 * s * M


def run_case(sw, dims, op, prec, dagger, apbc, r, masses, seed):
    import torch
    lat = Lattice(dims, apbc)
    Uh = ls.su3_links(dims, seed, ls.PLAQ_EPS)
    U = dev(Uh)
    U4 = lat.links(Uh)
    nc = 3 if op == sw.SW_OP_STAGGERED_WILSON else 12
    internal = (3,) if nc == 3 else (4, 3)
    W = None
    if nc == 3:
        W = torch.empty((lat.volume, 8, 3, 3), dtype=torch.complex128, device="cuda")
        sw.sw_hypercube_build(dims, U, W, apbc)
    ins = np.stack([ls.gaussian_source(dims, nc, seed + 10 + k).reshape((-1,) + internal)
                    for k in range(len(masses))])
    inp = dev(ins)
    out = torch.empty_like(inp)
    sw.dslash_apply_inner(dims, op, U, W, inp, out, masses, r, dagger, prec, apbc)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    worst = 0.0
    for k, m in enumerate(masses):
        f = lat.field(ins[k], internal)
        if nc == 3:
            ref = ops.sw_dslash(lat, U4, f, m, r, bool(dagger))
        else:
            ref = ops.wilson_dslash(lat, U4, f, m, r, bool(dagger))
        ref = lat.flat(ref, internal).reshape(lat.volume, -1)
        g = got[k].reshape(lat.volume, -1)
        M = np.sqrt((np.abs(ins[k].reshape(lat.volume, -1)) ** 2).sum(axis=1)).max()
        err = np.abs(g - ref).max()
        b = bound(nc, prec, r, m, M, np.abs(ref).max())
        assert err <= b, (op, prec, dagger, k, err, b)
        worst = max(worst, err / M)
    return worst


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dagger", [0, 1])
def test_inner_operator_matches_oracle(sw, op, prec, dagger):
    """6x6x4x6 (V = 864: several 128-site tiles and a ragged tail), antiperiodic
    time boundary, 5 systems of different masses (ragged register-blocking
    groups), r = 1 (spin-projected Wilson hops)."""
    run_case(sw, (6, 6, 4, 6), op, prec, dagger, True, 1.0, [0.05, 0.1, 0.2, 0.07, 0.3], 21)


@pytest.mark.parametrize("prec", [1, 2])
def test_inner_wilson_general_r(sw, prec):
    """Wilson at r = 0.75: the full 4-spinor hop of the inner kernels."""
    for dagger in (0, 1):
        run_case(sw, (4, 4, 2, 4), sw.SW_OP_WILSON, prec, dagger, False, 0.75, [0.1, 0.2, 0.05], 23)


@pytest.mark.parametrize("ns", [1, 2, 4])
def test_inner_every_register_blocking_width(sw, ns):
    """Both operators at each width of the inner stencils (7 systems: a
    ragged last group for widths 2 and 4), periodic boundaries."""
    old = (sw.sw_get_param(sw.SW_PARAM_NS_SW), sw.sw_get_param(sw.SW_PARAM_NS_WILSON))
    try:
        sw.sw_set_param(sw.SW_PARAM_NS_SW, ns)
        sw.sw_set_param(sw.SW_PARAM_NS_WILSON, ns)
        for op in (0, 1):
            for dagger in (0, 1):
                run_case(sw, (4, 6, 4, 4), op, sw.SW_PREC_F32_RELIABLE, dagger, False, 1.0,
                         [0.05, 0.1, 0.2, 0.07, 0.3, 0.02, 0.15], 25)
    finally:
        sw.sw_set_param(sw.SW_PARAM_NS_SW, old[0])
        sw.sw_set_param(sw.SW_PARAM_NS_WILSON, old[1])


def test_inner_rejects_f64_and_non_su3_half(sw):
    import torch
    dims = (4, 4, 4, 4)
    U = dev(ls.su3_links(dims, 1, ls.PLAQ_EPS))
    inp = dev(ls.gaussian_source(dims, 12, 3).reshape(1, -1, 4, 3))
    out = torch.empty_like(inp)
    with pytest.raises(sw.SWError) as e:
        sw.dslash_apply_inner(dims, sw.SW_OP_WILSON, U, None, inp, out, [0.1], 1.0, False, sw.SW_PREC_F64)
    assert e.value.code == -8
    with pytest.raises(sw.SWError) as e:
        sw.dslash_apply_inner(dims, sw.SW_OP_WILSON, U * 1.01, None, inp, out, [0.1], 1.0, False,
                              sw.SW_PREC_F16_RELIABLE)
    assert e.value.code == -8


@pytest.mark.parametrize("op", [0, 1])
def test_inner_operator_at_full_size(sw, op):
    """16^3x32 (mean plaquette 0.59) in the launch configuration of the bench's
    batches -- 12 staggered Wilson or 48 Wilson systems at the workload's four
    masses, the default width -- with the oracle's whole-field operator on the
    first and last system, both directions, FP32 storage."""
    import torch
    dims, masses = (16, 16, 16, 32), (0.02, 0.05, 0.1, 0.2)
    lat = Lattice(dims)
    Uh = ls.su3_links(dims, 0, ls.PLAQ_EPS, processes=8)
    U = dev(Uh)
    U4 = lat.links(Uh)
    nc, nsrc = (3, 3) if op == sw.SW_OP_STAGGERED_WILSON else (12, 12)
    internal = (3,) if nc == 3 else (4, 3)
    W = None
    if nc == 3:
        W = torch.empty((lat.volume, 8, 3, 3), dtype=torch.complex128, device="cuda")
        sw.sw_hypercube_build(dims, U, W)
    ms = [m for m in masses for _ in range(nsrc)]
    first = ls.gaussian_source(dims, nc, 31).reshape((-1,) + internal)
    last = ls.gaussian_source(dims, nc, 32).reshape((-1,) + internal)
    inp = torch.empty((len(ms),) + first.shape, dtype=torch.complex128, device="cuda")
    inp.normal_()
    inp[0] = dev(first)
    inp[-1] = dev(last)
    for dagger in (0, 1):
        out = torch.empty_like(inp)
        sw.dslash_apply_inner(dims, op, U, W, inp, out, ms, 1.0, dagger, sw.SW_PREC_F32_RELIABLE)
        torch.cuda.synchronize()
        for k, v in ((0, first), (len(ms) - 1, last)):
            f = lat.field(v, internal)
            ref = (ops.sw_dslash(lat, U4, f, ms[k], 1.0, bool(dagger)) if nc == 3 else
                   ops.wilson_dslash(lat, U4, f, ms[k], 1.0, bool(dagger)))
            ref = lat.flat(ref, internal).reshape(lat.volume, -1)
            g = out[k].cpu().numpy().reshape(lat.volume, -1)
            M = np.sqrt((np.abs(v.reshape(lat.volume, -1)) ** 2).sum(axis=1)).max()
            assert np.abs(g - ref).max() <= bound(nc, 1, 1.0, ms[k], M, np.abs(ref).max()), (op, dagger, k)
