"""cgne_solve_noalloc: the FP64 solve for callers that cannot call an allocator
while they run (runtimes whose device memory belongs to another allocator,
allocation-free latency loops), with its workspace in the library's static
device array.  Checked through the C ABI against cgne_solve on calls in a row
-- a staggered Wilson solve, a larger Wilson solve, then a smaller staggered
Wilson solve from a non-zero initial guess, so that the shared array holds a
larger call's leftovers -- within the solution tolerance of the other GPU
tests (1e-6 relative), plus the size limit.  Kept last in collection order so
that a -x run has already run every other test."""
import ctypes

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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def c_solve(sw, fn, dims, op, U, W, chi, x, mass, tol):
    """Call an entry point through ctypes: fn is 'cgne_solve' or 'cgne_solve_noalloc'
    (x holds the initial guess on entry and the solution on exit)."""
    import torch
    from paper_1312_3265_gb300._binding import Lattice, _Info
    L = sw.lib()
    lat = Lattice((ctypes.c_int * 4)(*dims), 0)
    info = _Info()
    stream = torch.cuda.current_stream().cuda_stream
    Wp = W.data_ptr() if W is not None else None
    if fn == "cgne_solve":
        rc = L.cgne_solve(ctypes.byref(lat), op, U.data_ptr(), Wp, chi.data_ptr(), x.data_ptr(), mass, 1.0, tol,
                          100000, sw.SW_PREC_F64, ctypes.byref(info), stream)
    else:
        rc = L.cgne_solve_noalloc(ctypes.byref(lat), op, U.data_ptr(), Wp, chi.data_ptr(), x.data_ptr(), mass, 1.0,
                                  tol, 100000, ctypes.byref(info), stream)
    torch.cuda.synchronize()
    return rc, info


def problem(sw, dims, op, seed):
    import torch
    V = ls.volume(dims)
    U = dev(ls.su3_links(dims, seed, ls.PLAQ_EPS))
    W = None
    nc = 3 if op == sw.SW_OP_STAGGERED_WILSON else 12
    if nc == 3:
        W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
        sw.sw_hypercube_build(dims, U, W)
    chi = dev(ls.gaussian_source(dims, nc, seed + 1))
    return U, W, chi


def test_noalloc_matches_cgne_solve_in_a_row(sw):
    import torch
    # calls in a row: different operators and sizes, the last one smaller than
    # the one before it and started from a non-zero guess
    cases = [((4, 4, 4, 4), sw.SW_OP_STAGGERED_WILSON, 0.05, False), ((6, 4, 4, 6), sw.SW_OP_WILSON, 0.1, False),
             ((4, 4, 2, 4), sw.SW_OP_STAGGERED_WILSON, 0.07, True)]
    for dims, op, mass, guess in cases:
        U, W, chi = problem(sw, dims, op, 3)
        x0 = dev(ls.gaussian_source(dims, chi.shape[-1], 17)) if guess else None
        x_ref = x0.clone() if guess else torch.zeros_like(chi)
        rc, ref_info = c_solve(sw, "cgne_solve", dims, op, U, W, chi, x_ref, mass, 1e-10)
        assert rc == sw.SW_OK
        x = x0.clone() if guess else torch.zeros_like(chi)
        rc, info = c_solve(sw, "cgne_solve_noalloc", dims, op, U, W, chi, x, mass, 1e-10)
        assert rc == sw.SW_OK and info.status == sw.SW_OK
        assert info.true_rel_resid <= 1e-10
        a, b = x.cpu().numpy(), x_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-6
        assert abs(info.iters - ref_info.iters) <= 1


def test_noalloc_rejects_lattices_beyond_the_scratch(sw):
    import torch
    dims = (16, 16, 16, 32)  # Wilson needs 768 B/site: 96 MiB > 32 MiB
    V = ls.volume(dims)
    U = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    chi = torch.zeros((V, 4, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(chi)
    rc, _ = c_solve(sw, "cgne_solve_noalloc", dims, sw.SW_OP_WILSON, U, None, chi, x, 0.1, 1e-8)
    assert rc == -8
