"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no Dirac-operator or solver arithmetic.  It only makes
inputs: SU(3) gauge links, fermion sources and random gauge transformations,
all drawn from a counter-based generator so that any subset of sites can be
regenerated independently and identically on any machine.

Canonical layouts (the ones the C ABI takes):
  site index  n = x0 + L0*(x1 + L1*(x2 + L2*x3)),  x3 = time
  links       U[n][mu][a][b]  complex128, mu = 0..3 (U_mu(x) joins x -> x+mu)
  colour vec  psi[n][a]       complex128 (staggered-type, one component per site)
  spinor      psi[n][s][a]    complex128 (Wilson, spin s = 0..3, colour a)

Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC11), written here from its published round
function and checked against the published known-answer vectors in the tests.
Normals come from the Box-Muller transform of pairs of uniforms.

Gauge links follow the workloads of the cost comparison (Sec. 3 of the paper:
16^3x32 quenched backgrounds at beta = 6, mean plaquette about 0.59): the
backgrounds are replaced by U = exp(i eps H), H = sum_a theta_a lambda_a with
theta_a ~ N(0,1) and lambda_a the Gell-Mann matrices, re-unitarised to SU(3).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10", "uniforms", "normals", "gell_mann",
    "volume", "site_coords", "su3_links", "reunitarize", "plaquette",
    "tune_eps", "PLAQ_EPS", "LINK_EPS_SMALL",
    "point_source", "z2_source", "gaussian_source", "haar_su3",
    "STREAM_LINKS", "STREAM_GAUSS", "STREAM_Z2", "STREAM_GAUGE_XFORM",
]

# Philox-4x32-10 multipliers and Weyl key increments (published constants).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

# Stream tags: third counter word, so different input kinds never overlap.
STREAM_LINKS = 1
STREAM_GAUSS = 2
STREAM_Z2 = 3
STREAM_GAUGE_XFORM = 4

# eps for which seed-0 links give a mean plaquette of 0.59 (tuned by
# tune_eps() on an 8^4 lattice, seed 0; re-checked by the tests).
PLAQ_EPS = 0.2190
# eps of the small 4^4 staggered Wilson workload (fixed, not tuned).
LINK_EPS_SMALL = 0.3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32-10 on arrays of 32-bit counter words; returns 4 uint32 arrays."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    shape = np.broadcast_shapes(*(v.shape for v in c))
    c = [np.broadcast_to(v, shape).copy() for v in c]
    ka = np.uint64(k0) & _MASK
    kb = np.uint64(k1) & _MASK
    for rnd in range(10):
        if rnd:
            ka = (ka + _W0) & _MASK
            kb = (kb + _W1) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ ka, lo1, hi0 ^ c[3] ^ kb, lo0]
    return [v.astype(np.uint32) for v in c]


def _key(seed):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def uniforms(n_index, stream, seed):
    """Four uniforms in (0,1) per counter index: array shape (..., 4)."""
    n = np.asarray(n_index, dtype=np.uint64)
    k0, k1 = _key(seed)
    words = philox4x32_10(n & _MASK, n >> np.uint64(32), np.uint64(stream), 0, k0, k1)
    u = np.stack(words, axis=-1).astype(np.float64)
    return (u + 0.5) * (1.0 / 4294967296.0)


def normals(n_index, stream, seed):
    """Four standard normals per counter index (Box-Muller on two uniform pairs)."""
    u = uniforms(n_index, stream, seed)
    rad0 = np.sqrt(-2.0 * np.log(u[..., 0]))
    rad1 = np.sqrt(-2.0 * np.log(u[..., 2]))
    ang0 = 2.0 * np.pi * u[..., 1]
    ang1 = 2.0 * np.pi * u[..., 3]
    return np.stack([rad0 * np.cos(ang0), rad0 * np.sin(ang0),
                     rad1 * np.cos(ang1), rad1 * np.sin(ang1)], axis=-1)


def gell_mann():
    """The eight Gell-Mann matrices, shape (8, 3, 3), Tr(l_a l_b) = 2 delta_ab."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return lam


def volume(dims):
    d = [int(v) for v in dims]
    return d[0] * d[1] * d[2] * d[3]


def site_coords(dims, n=None):
    """Coordinates (x0, x1, x2, x3) of site index n (all sites if n is None)."""
    if n is None:
        n = np.arange(volume(dims))
    n = np.asarray(n)
    x0 = n % dims[0]
    n1 = n // dims[0]
    x1 = n1 % dims[1]
    n2 = n1 // dims[1]
    x2 = n2 % dims[2]
    x3 = n2 // dims[2]
    return x0, x1, x2, x3


def reunitarize(M):
    """Project (..., 3, 3) matrices onto SU(3): Gram-Schmidt on rows 0 and 1,
    third row the complex conjugate of their cross product."""
    r0 = M[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = M[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def su3_links(dims, seed, eps, sites=None, processes=1):
    """Gauge links U[n][mu] = reunitarize(exp(i eps sum_a theta_a lambda_a)).

    theta_a(n, mu) ~ N(0,1) from Philox counter index 2*(4 n + mu) + j, j = 0,1,
    stream STREAM_LINKS, key = seed.  `sites` selects a subset of site indices
    (same values as the full field at those sites).  Returns (nsites, 4, 3, 3).
    processes > 1 splits the sites over that many worker processes (spawned,
    writing into shared memory); the values are the same.
    """
    if sites is None and processes > 1 and volume(dims) >= 65536:
        return _su3_links_parallel(dims, seed, eps, processes)
    if sites is None:
        sites = np.arange(volume(dims), dtype=np.int64)
    sites = np.asarray(sites, dtype=np.int64)
    base = (sites[:, None] * 4 + np.arange(4)[None, :]) * 2  # (ns, 4)
    z = np.concatenate([normals(base, STREAM_LINKS, seed),
                        normals(base + 1, STREAM_LINKS, seed)], axis=-1)  # (ns,4,8)
    H = np.einsum("sma,aij->smij", z, gell_mann())
    w, V = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    U = np.einsum("smik,smk,smjk->smij", V, ph, np.conj(V))
    return reunitarize(U)


def _links_into(name, shape, dims, seed, eps, lo, hi):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        step = 1 << 16
        for a in range(lo, hi, step):
            b = min(hi, a + step)
            out[a:b] = su3_links(dims, seed, eps, sites=np.arange(a, b, dtype=np.int64))
    finally:
        shm.close()


def _su3_links_parallel(dims, seed, eps, processes):
    import multiprocessing as mp
    from multiprocessing import shared_memory
    V = volume(dims)
    shape = (V, 4, 3, 3)
    shm = shared_memory.SharedMemory(create=True, size=V * 4 * 9 * 16)
    try:
        bounds = np.linspace(0, V, processes * 4 + 1).astype(np.int64)
        ctx = mp.get_context("spawn")  # safe after CUDA has been initialised in the parent
        with ctx.Pool(processes) as pool:
            pool.starmap(_links_into, [(shm.name, shape, tuple(dims), seed, eps, int(bounds[i]), int(bounds[i + 1]))
                                       for i in range(len(bounds) - 1)])
        return np.array(np.ndarray(shape, dtype=np.complex128, buffer=shm.buf))
    finally:
        shm.close()
        shm.unlink()


def _shift_index(dims, mu, step=1):
    """Index map n -> n + step*mu_hat (periodic)."""
    x = list(site_coords(dims))
    x[mu] = (x[mu] + step) % dims[mu]
    return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))


def plaquette(U, dims):
    """Mean plaquette (1/3) Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+,
    averaged over sites and the 6 planes."""
    tot = 0.0
    for mu in range(4):
        fmu = _shift_index(dims, mu)
        for nu in range(mu + 1, 4):
            fnu = _shift_index(dims, nu)
            P = (U[:, mu] @ U[fmu, nu]) @ np.conj(np.swapaxes(U[fnu, mu], -1, -2)) \
                @ np.conj(np.swapaxes(U[:, nu], -1, -2))
            tot += np.mean(np.real(np.trace(P, axis1=-2, axis2=-1))) / 3.0
    return tot / 6.0


def tune_eps(target=0.59, dims=(8, 8, 8, 8), seed=0, lo=0.05, hi=0.5, iters=40):
    """Bisection on eps so that the seed's mean plaquette equals `target`."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if plaquette(su3_links(dims, seed, mid), dims) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def point_source(dims, ncomp, alpha, site=0):
    """Unit source: 1 at `site`, flattened component alpha (colour, or spin*3+colour)."""
    v = np.zeros((volume(dims), ncomp), dtype=np.complex128)
    v[site, alpha] = 1.0
    return v


def gaussian_source(dims, ncomp, seed):
    """Complex Gaussian source, Re and Im ~ N(0,1) per component."""
    n = np.arange(volume(dims) * ncomp, dtype=np.int64)
    z = normals(n, STREAM_GAUSS, seed)
    return (z[:, 0] + 1j * z[:, 1]).reshape(volume(dims), ncomp)


def z2_source(dims, ncomp, seed):
    """Real Z2 noise: +-1 in the real part of every component."""
    n = np.arange(volume(dims) * ncomp, dtype=np.int64)
    u = uniforms(n, STREAM_Z2, seed)[:, 0]
    return np.where(u < 0.5, 1.0, -1.0).astype(np.complex128).reshape(volume(dims), ncomp)


def haar_su3(dims, seed):
    """Random SU(3) matrix per site (QR of a complex Gaussian, phase-fixed so
    the unitary factor is Haar on U(3), then divided by a cube root of det)."""
    n = np.arange(volume(dims), dtype=np.int64)
    z = np.concatenate([normals(n * 5 + k, STREAM_GAUGE_XFORM, seed) for k in range(5)],
                       axis=-1)[:, :18]
    G = (z[:, 0::2] + 1j * z[:, 1::2]).reshape(-1, 3, 3)
    Q, R = np.linalg.qr(G)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]
