"""Dense matrices of the operators on small lattices, for spectra, condition
numbers kappa = lmax/lmin of (D+m)^+(D+m) (Sec. 3) and direct LU solves."""
from __future__ import annotations

import numpy as np

from . import operators as ops
from .lattice import Lattice


def matrix(apply, lat: Lattice, internal):
    """Dense N x N matrix M with M e_j = apply(e_j), N = V * prod(internal).

    `apply` maps a batch of fields (N, L3, L2, L1, L0, *internal) to the same shape.
    """
    nloc = int(np.prod(internal))
    N = lat.volume * nloc
    E = np.eye(N, dtype=np.complex128).reshape((N,) + lat.shape + tuple(internal))
    out = apply(E).reshape(N, N)
    return out.T.copy()


def sw_matrix(lat, U4, mass, r=1.0, dagger=False):
    return matrix(lambda v: ops.sw_dslash(lat, U4, v, mass, r, dagger), lat, (3,))


def wilson_matrix(lat, U4, mass, r=1.0, dagger=False):
    return matrix(lambda v: ops.wilson_dslash(lat, U4, v, mass, r, dagger), lat, (4, 3))


def normal_spectrum(M):
    """Eigenvalues of M^+ M (ascending)."""
    return np.linalg.eigvalsh(M.conj().T @ M)


def condition_number(M):
    ev = normal_spectrum(M)
    return ev[-1] / ev[0]


def direct_solve(M, chi_flat):
    """psi = M^{-1} chi by LU (numpy.linalg.solve)."""
    return np.linalg.solve(M, chi_flat)
