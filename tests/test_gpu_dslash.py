"""GPU parity of the FP64 operator kernels against the oracle, through the C ABI.

Tolerance: 1e-12 relative (max-norm of the difference over max-norm of the
oracle result) for FP64 matvecs; hypercube transports 1e-13.  On lattices too
large for the whole-field oracle the same measure is taken over sampled
sites: the largest difference at the samples over the largest oracle value at
the samples (the rounding error of a site scales with its inputs, not with
its own output, which can be small).
"""
import numpy as np
import pytest

import lattice_synth as ls
from oracle import Lattice, operators as ops, site

pytestmark = pytest.mark.gpu

TOL = 1e-12
# several tiles and ragged tails (V = 864, 1200 are not multiples of 128),
# L = 2 extents (neighbours alias), mixed extents
LATTICES = [(4, 4, 4, 4), (6, 6, 4, 6), (2, 2, 2, 2), (2, 4, 6, 2), (10, 4, 6, 10), (8, 8, 8, 8)]


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


def rand_vec(V, nc, seed):
    return ls.gaussian_source((V, 1, 1, 1), nc, seed).reshape(V, nc)


def relerr(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


class Sampled:
    """Max-norm relative error over sampled sites (see the module docstring)."""

    def __init__(self):
        self.diff, self.scale = 0.0, 0.0

    def add(self, got, want):
        self.diff = max(self.diff, float(np.abs(got - want).max()))
        self.scale = max(self.scale, float(np.abs(want).max()))

    def rel(self):
        return self.diff / self.scale


def make_fields(sw, dims, seed=3, eps=0.5):
    import torch
    V = ls.volume(dims)
    Uh = ls.su3_links(dims, seed, eps)
    U = dev(Uh)
    W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
    sw.sw_hypercube_build(dims, U, W)
    return Uh, U, W


@pytest.mark.parametrize("dims", LATTICES)
def test_hypercube_transports(sw, dims):
    import torch
    Uh, U, W = make_fields(sw, dims)
    torch.cuda.synchronize()
    lat = Lattice(dims)
    want = ops.hypercube_all(lat, lat.links(Uh))  # (8, L3..L0, 3, 3)
    want = np.moveaxis(want.reshape(8, lat.volume, 3, 3), 0, 1)
    assert relerr(W.cpu().numpy(), want) < 1e-13


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("apbc", [False, True])
def test_sw_dslash(sw, dims, apbc):
    import torch
    Uh, U, W = make_fields(sw, dims)
    lat = Lattice(dims, apbc)
    U4 = lat.links(Uh)
    psi_h = rand_vec(lat.volume, 3, 5)
    psi = dev(psi_h)
    out = torch.empty_like(psi)
    for mass, r, dag in ((0.05, 1.0, False), (0.05, 1.0, True), (0.3, 0.7, False), (0.0, 1.0, True)):
        sw.sw_dslash_apply(dims, U, W, psi, out, mass, r, dag, apbc)
        torch.cuda.synchronize()
        want = lat.flat(ops.sw_dslash(lat, U4, lat.field(psi_h, (3,)), mass, r, dag), (3,))
        assert relerr(out.cpu().numpy(), want) < TOL, (mass, r, dag)


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("apbc", [False, True])
def test_wilson_dslash(sw, dims, apbc):
    import torch
    Uh = ls.su3_links(dims, 4, 0.5)
    U = dev(Uh)
    lat = Lattice(dims, apbc)
    U4 = lat.links(Uh)
    psi_h = rand_vec(lat.volume, 12, 6).reshape(lat.volume, 4, 3)
    psi = dev(psi_h)
    out = torch.empty_like(psi)
    for mass, r, dag in ((0.05, 1.0, False), (0.05, 1.0, True), (0.2, 0.8, False), (0.2, 0.8, True)):
        sw.wilson_dslash_apply(dims, U, psi, out, mass, r, dag, apbc)
        torch.cuda.synchronize()
        want = lat.flat(ops.wilson_dslash(lat, U4, lat.field(psi_h, (4, 3)), mass, r, dag), (4, 3))
        assert relerr(out.cpu().numpy(), want) < TOL, (mass, r, dag)


def test_full_size_sampled_sites(sw):
    """16^3x32 (the paper's lattice, mean plaquette 0.59 links): sampled output
    sites against the one-site oracle, antiperiodic in time."""
    import torch
    dims = (16, 16, 16, 32)
    V = ls.volume(dims)
    Uh, U, W = make_fields(sw, dims, seed=0, eps=ls.PLAQ_EPS)
    psi_h = rand_vec(V, 3, 7)
    spn_h = rand_vec(V, 12, 8).reshape(V, 4, 3)
    psi, spn = dev(psi_h), dev(spn_h)
    o1, o2 = torch.empty_like(psi), torch.empty_like(spn)
    sw.sw_dslash_apply(dims, U, W, psi, o1, 0.02, 1.0, True, True)
    sw.wilson_dslash_apply(dims, U, spn, o2, 0.02, 1.0, False, True)
    torch.cuda.synchronize()
    a, b = o1.cpu().numpy(), o2.cpu().numpy()
    rng = np.random.default_rng(0)
    sites = np.concatenate([[0, V - 1, 16 * 16 * 16 * 31, 15], rng.integers(0, V, 28)])
    es, ew = Sampled(), Sampled()
    for n in sites:
        n = int(n)
        es.add(a[n], site.sw_dslash_site(Uh, psi_h, dims, n, 0.02, 1.0, True, True))
        ew.add(b[n], site.wilson_dslash_site(Uh, spn_h, dims, n, 0.02, 1.0, False, True))
    assert es.rel() < TOL and ew.rel() < TOL, (es.rel(), ew.rel())


def test_abi_rejects_bad_arguments(sw):
    import torch
    dims = (4, 4, 4, 4)
    V = 256
    U = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    W = torch.zeros((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
    v = torch.zeros((V, 3), dtype=torch.complex128, device="cuda")
    o = torch.zeros_like(v)
    with pytest.raises(sw.SWError) as e:
        sw.sw_dslash_apply((4, 4, 4, 3), U, W, v, o, 0.1)
    assert e.value.code == -1
    with pytest.raises(sw.SWError) as e:
        sw.sw_dslash_apply(dims, U, W, None, o, 0.1)
    assert e.value.code == -2
    with pytest.raises(sw.SWError) as e:
        sw.sw_dslash_apply(dims, U, W, v.data_ptr() + 8, o, 0.1)
    assert e.value.code == -3
    host = np.zeros((V, 3), dtype=np.complex128)
    with pytest.raises(sw.SWError) as e:
        sw.sw_dslash_apply(dims, U, W, host.ctypes.data, o, 0.1)
    assert e.value.code == -8
    with pytest.raises(sw.SWError) as e:  # in and out overlap
        sw.sw_dslash_apply(dims, U, W, v, v, 0.1)
    assert e.value.code == -8


def test_large_lattice_sampled_sites(sw):
    """24^3x48 (the batched multi-source workload's lattice; FP32 links no longer
    fit in L2): sampled output sites of both FP64 operators against the one-site
    oracle, periodic in time."""
    import torch
    dims = (24, 24, 24, 48)
    V = ls.volume(dims)
    Uh = ls.su3_links(dims, 0, ls.PLAQ_EPS, processes=8)
    U = dev(Uh)
    W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
    sw.sw_hypercube_build(dims, U, W)
    psi_h = rand_vec(V, 3, 17)
    spn_h = rand_vec(V, 12, 18).reshape(V, 4, 3)
    psi, spn = dev(psi_h), dev(spn_h)
    o1, o2 = torch.empty_like(psi), torch.empty_like(spn)
    sw.sw_dslash_apply(dims, U, W, psi, o1, 0.05, 1.0, False)
    sw.wilson_dslash_apply(dims, U, spn, o2, 0.05, 1.0, True)
    torch.cuda.synchronize()
    a, b = o1.cpu().numpy(), o2.cpu().numpy()
    rng = np.random.default_rng(1)
    es, ew = Sampled(), Sampled()
    for n in np.concatenate([[0, V - 1], rng.integers(0, V, 14)]):
        n = int(n)
        es.add(a[n], site.sw_dslash_site(Uh, psi_h, dims, n, 0.05, 1.0, False, False))
        ew.add(b[n], site.wilson_dslash_site(Uh, spn_h, dims, n, 0.05, 1.0, True, False))
    assert es.rel() < TOL and ew.rel() < TOL, (es.rel(), ew.rel())


def test_largest_lattices_sampled_sites(sw):
    """The large-volume workloads' lattices: 48^3x96 staggered Wilson (10.6 M
    sites, periodic) and 32^3x64 Wilson (antiperiodic): sampled output sites of
    the FP64 operators -- the ones that decide convergence -- against the
    one-site oracle, including the first and last sites and both time
    boundaries (complex-element indices beyond 2^24)."""
    import torch
    for dims, op in (((48, 48, 48, 96), "sw"), ((32, 32, 32, 64), "wilson")):
        V = ls.volume(dims)
        Uh = ls.su3_links(dims, 2, ls.PLAQ_EPS, processes=16)
        U = dev(Uh)
        rng = np.random.default_rng(3)
        slab = dims[0] * dims[1] * dims[2]
        sites = np.concatenate([[0, V - 1, slab - 1, V - slab, (V // 2) | 1], rng.integers(0, V, 10)])
        if op == "sw":
            W = torch.empty((V, 8, 3, 3), dtype=torch.complex128, device="cuda")
            sw.sw_hypercube_build(dims, U, W)
            psi_h = rand_vec(V, 3, 27)
            psi = dev(psi_h)
            out = torch.empty_like(psi)
            sw.sw_dslash_apply(dims, U, W, psi, out, 0.01, 1.0, False)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            del W, out
            e = Sampled()
            for n in sites:
                e.add(got[int(n)], site.sw_dslash_site(Uh, psi_h, dims, int(n), 0.01, 1.0, False, False))
            assert e.rel() < TOL, (op, e.rel())
        else:
            spn_h = rand_vec(V, 12, 28).reshape(V, 4, 3)
            spn = dev(spn_h)
            out = torch.empty_like(spn)
            sw.wilson_dslash_apply(dims, U, spn, out, 0.01, 1.0, True, True)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            del out
            e = Sampled()
            for n in sites:
                e.add(got[int(n)], site.wilson_dslash_site(Uh, spn_h, dims, int(n), 0.01, 1.0, True, True))
            assert e.rel() < TOL, (op, e.rel())
        del U
        torch.cuda.empty_cache()
