"""One-site evaluation of the operators with explicit loops.

Used to check sampled output sites of lattices too large for the whole-field
oracle.  Inputs are canonical flat arrays: U (V,4,3,3), psi (V,3) or (V,4,3).
Each output site is computed from its own definition (Sec. 1-3 readings as in
operators.py), path by path, with no precomputed hypercube transport.
"""
from __future__ import annotations

import numpy as np

from .lattice import PERMUTATIONS, hypercube_vectors
from .operators import gamma_matrices


def coords(dims, n):
    x0 = n % dims[0]
    n //= dims[0]
    x1 = n % dims[1]
    n //= dims[1]
    x2 = n % dims[2]
    x3 = n // dims[2]
    return [x0, x1, x2, x3]


def index(dims, x):
    return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * x[3]))


def step(dims, x, mu, s, antiperiodic_t):
    """Neighbour coordinates x + s*mu and the fermion boundary sign of the hop."""
    y = list(x)
    y[mu] += s
    sign = 1.0
    if y[mu] < 0 or y[mu] >= dims[mu]:
        y[mu] %= dims[mu]
        if mu == 3 and antiperiodic_t:
            sign = -1.0
    return y, sign


def link(U, dims, y, mu, s):
    """Link for a step s*mu from y: U_mu(y) or U_mu(y-mu)^+."""
    if s > 0:
        return U[index(dims, y), mu]
    z, _ = step(dims, y, mu, -1, False)
    return np.conj(U[index(dims, z), mu]).T


def hypercube_site(U, dims, n, svec):
    """W(x, s) at one site: average over the 24 orderings of the path product."""
    x0 = coords(dims, n)
    W = np.zeros((3, 3), dtype=np.complex128)
    for perm in PERMUTATIONS:
        M = np.eye(3, dtype=np.complex128)
        y = list(x0)
        for mu in perm:
            M = M @ link(U, dims, y, mu, svec[mu])
            y, _ = step(dims, y, mu, svec[mu], False)
        W += M
    return W / 24.0


def sw_dslash_site(U, psi, dims, n, mass, r=1.0, dagger=False, antiperiodic_t=False):
    """((D_SW + m) psi)(x) at site n (adjoint if dagger)."""
    x = coords(dims, n)
    psi = np.asarray(psi).reshape(-1, 3)
    dst = np.zeros(3, dtype=np.complex128)
    for mu in range(4):
        eta = (-1) ** (sum(x[:mu]) % 2)
        yf, sf = step(dims, x, mu, +1, antiperiodic_t)
        yb, sb = step(dims, x, mu, -1, antiperiodic_t)
        dst += eta * (sf * U[n, mu] @ psi[index(dims, yf)]
                      - sb * np.conj(U[index(dims, yb), mu]).T @ psi[index(dims, yb)])
    dst *= 0.5
    g = np.zeros(3, dtype=np.complex128)
    for svec in hypercube_vectors(False):
        y = list(x)
        sign = 1.0
        for mu in range(4):
            y, sg = step(dims, y, mu, svec[mu], antiperiodic_t)
            sign *= sg
        g += sign * hypercube_site(U, dims, n, svec) @ psi[index(dims, y)]
    g *= (-1) ** ((x[1] + x[3]) % 2) / 16.0  # eps(x) eta5(x) = (-1)^(x1+x3)
    sgn = -1.0 if dagger else 1.0
    return sgn * dst + r * (psi[n] - g) + mass * psi[n]


def wilson_dslash_site(U, psi, dims, n, mass, r=1.0, dagger=False, antiperiodic_t=False):
    """((D_W + m) psi)(x) at site n (adjoint if dagger); psi shaped (V,4,3)."""
    G, _ = gamma_matrices()
    sg = -1.0 if dagger else 1.0
    x = coords(dims, n)
    psi = np.asarray(psi).reshape(-1, 4, 3)
    out = (4.0 * r + mass) * psi[n]
    one = np.eye(4)
    for mu in range(4):
        yf, sf = step(dims, x, mu, +1, antiperiodic_t)
        yb, sb = step(dims, x, mu, -1, antiperiodic_t)
        f = sf * (U[n, mu] @ psi[index(dims, yf)].T).T
        b = sb * (np.conj(U[index(dims, yb), mu]).T @ psi[index(dims, yb)].T).T
        out = out - 0.5 * ((r * one - sg * G[mu]) @ f + (r * one + sg * G[mu]) @ b)
    return out
