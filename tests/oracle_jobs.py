"""Oracle computations for the full-size GPU tests, run in spawned worker
processes (started before, or independently of, any CUDA context) so that the
slow FP64 numpy oracle works while the GPU tests run.  Every function here
calls only oracle/ and lattice_synth/ (the seeded input generator)."""
from __future__ import annotations

import numpy as np

import lattice_synth as ls
from oracle import Lattice, operators as ops
from oracle.cg import cgne


def _operator(lat, U4, nc, mass, r=1.0, W16=None):
    if nc == 3:
        return (lambda v: ops.sw_dslash(lat, U4, v, mass, r, False, W16),
                lambda v: ops.sw_dslash(lat, U4, v, mass, r, True, W16))
    return (lambda v: ops.wilson_dslash(lat, U4, v, mass, r, False),
            lambda v: ops.wilson_dslash(lat, U4, v, mass, r, True))


def point_solution(dims, seed, eps, nc, alpha, mass, tol):
    """The oracle's CGNE solution (Eq. 2, textbook CG from x0 = 0) for the
    point source at the origin with component alpha, on the links of
    (seed, eps).  Staggered Wilson uses the transport form of Gamma55 (the
    oracle's hypercube transports, pinned to the literal symmetrised product).
    Returns (x flat (V, nc), iterations, true relative residual, the first
    iteration whose iterated residual was <= 1e-8)."""
    lat = Lattice(dims)
    U4 = lat.links(ls.su3_links(dims, seed, eps))
    internal = (3,) if nc == 3 else (4, 3)
    W16 = ops.hypercube_all(lat, U4, stored_only=False) if nc == 3 else None
    D, Dd = _operator(lat, U4, nc, mass, 1.0, W16)
    chi = lat.field(ls.point_source(dims, nc, alpha).reshape((-1,) + internal), internal)
    x, info = cgne(D, Dd, chi, tol, 100000)
    k8 = next(k for k, h in enumerate(info["history"]) if h <= 1e-8)
    return lat.flat(x, internal).reshape(lat.volume, nc), info["iters"], info["true_rel_resid"], k8


def normal_residual(dims, seed, eps, nc, mass, chi_flat, x_flat):
    """|b - A x| / |b| with A = (D+m)^+(D+m), b = (D+m)^+ chi, by the oracle's
    literal operators."""
    lat = Lattice(dims)
    U4 = lat.links(ls.su3_links(dims, seed, eps))
    internal = (3,) if nc == 3 else (4, 3)
    D, Dd = _operator(lat, U4, nc, mass)
    chi = lat.field(np.asarray(chi_flat).reshape((-1,) + internal), internal)
    x = lat.field(np.asarray(x_flat).reshape((-1,) + internal), internal)
    b = Dd(chi)
    r = b - Dd(D(x))
    return float(np.linalg.norm(r) / np.linalg.norm(b))
