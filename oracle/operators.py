"""Lattice Dirac operators of the cost comparison, written from their definitions.

All functions take fields in the oracle's lattice shape (see lattice.py) with
any number of leading batch axes, and return new arrays.  FP64/complex128.

Staggered Wilson (2 flavours; Sec. 1-2 of the paper, operator of Adams,
PLB 699 (2011) 394, which the paper cites instead of printing it):
    (D_st psi)(x)   = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^+ psi(x-mu)]
    C_mu            = (V_mu + V_mu^+)/2
    Gamma55         = eps(x) eta5(x) (1/24) sum_{sigma in S4} C_s0 C_s1 C_s2 C_s3
    D_SW + m        = D_st + r (1 - Gamma55) + m
The site couples to 8 one-hop and 16 hypercube-corner neighbours (Sec. 3,
"8+16").  D_st is anti-Hermitian and Gamma55 Hermitian, so the adjoint is
D_SW^+ + m = -D_st + r(1 - Gamma55) + m.

Wilson (the 1392 flop/site operator of Eq. 4):
    (D_W psi)(x) = (4r + m) psi(x)
                   - 1/2 sum_mu [(r - g_mu) U_mu(x) psi(x+mu) + (r + g_mu) U_mu(x-mu)^+ psi(x-mu)]
with Hermitian gamma matrices in the DeGrand-Rossi basis; the adjoint flips
the sign of every g_mu.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice, PERMUTATIONS, hypercube_vectors

# ---------------------------------------------------------------- gammas


def gamma_matrices():
    """DeGrand-Rossi gamma_0..3 (x, y, z, t) and gamma5 = g0 g1 g2 g3."""
    i = 1j
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    g[0] = [[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]]
    g[1] = [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]]
    g[2] = [[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]]
    g[3] = [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]]
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


# ---------------------------------------------------------------- hops


def _dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def _mul(A, psi, nint):
    """Colour matrix times field: A(x) psi(x)."""
    if nint == 1:
        return np.einsum("...ab,...b->...a", A, psi)
    return np.einsum("...ab,...sb->...sa", A, psi)


def hop_fwd(lat: Lattice, U, psi, mu, nint=1):
    """(V_mu psi)(x) = U_mu(x) psi(x + mu)."""
    return _mul(U[mu], lat.shift(psi, mu, +1, nint), nint)


def hop_bwd(lat: Lattice, U, psi, mu, nint=1):
    """(V_mu^+ psi)(x) = U_mu(x - mu)^+ psi(x - mu)."""
    return lat.shift(_mul(_dag(U[mu]), psi, nint), mu, -1, nint)


def _bc(phase, nint):
    return phase.reshape(phase.shape + (1,) * nint)


# ---------------------------------------------------------------- staggered Wilson


def staggered(lat: Lattice, U, psi):
    """D_st psi = 1/2 sum_mu eta_mu (V_mu - V_mu^+) psi."""
    out = np.zeros_like(psi)
    for mu in range(4):
        out += _bc(lat.eta(mu), 1) * (hop_fwd(lat, U, psi, mu) - hop_bwd(lat, U, psi, mu))
    return 0.5 * out


def c_op(lat: Lattice, U, psi, mu):
    """C_mu psi = (V_mu + V_mu^+) psi / 2."""
    return 0.5 * (hop_fwd(lat, U, psi, mu) + hop_bwd(lat, U, psi, mu))


def gamma55_literal(lat: Lattice, U, psi):
    """Gamma55 psi = eps eta5 (1/24) sum over the 24 orderings of C C C C psi."""
    acc = np.zeros_like(psi)
    for perm in PERMUTATIONS:
        v = psi
        for mu in reversed(perm):  # C_p0 C_p1 C_p2 C_p3 psi: rightmost acts first
            v = c_op(lat, U, v, mu)
        acc += v
    return _bc(lat.epsilon() * lat.eta5(), 1) * acc / 24.0


def hypercube_transport(lat: Lattice, U, svec):
    """W(x, s) = (1/24) sum_sigma of the 4-link path product from x to x+s.

    The path in ordering sigma steps s_mu along mu for mu = sigma_0, ..., sigma_3;
    a step +mu from y contributes U_mu(y), a step -mu contributes U_mu(y-mu)^+.
    Pure gauge transport: no fermion boundary sign.  Shape (L3,L2,L1,L0,3,3).
    """
    fwd = U
    bwd = [np.roll(_dag(U[mu]), 1, axis=-(3 + mu)) for mu in range(4)]  # U_mu(y-mu)^+
    W = np.zeros(lat.shape + (3, 3), dtype=np.complex128)
    for perm in PERMUTATIONS:
        M = np.broadcast_to(np.eye(3, dtype=np.complex128), lat.shape + (3, 3))
        off = [0, 0, 0, 0]
        for mu in perm:
            L = fwd[mu] if svec[mu] > 0 else bwd[mu]
            M = M @ lat.shift_links(L, off)
            off[mu] += svec[mu]
        W = W + M
    return W / 24.0


def hypercube_all(lat: Lattice, U, stored_only=True):
    """W for the stored displacements (8, s3 = +1) or all 16, stacked on axis 0."""
    return np.stack([hypercube_transport(lat, U, s)
                     for s in hypercube_vectors(stored_only)])


def shift_multi(lat: Lattice, psi, svec, nint=1):
    """psi(x + s), boundary signs included."""
    for mu in range(4):
        psi = lat.shift(psi, mu, svec[mu], nint)
    return psi


def gamma55_from_transport(lat: Lattice, W16, psi):
    """Gamma55 psi = eps eta5 (1/16) sum_{s in {+-1}^4} W(x,s) psi(x+s), with W16
    the 16 transports from hypercube_all(..., stored_only=False)."""
    acc = np.zeros_like(psi)
    for k, s in enumerate(hypercube_vectors(False)):
        acc += _mul(W16[k], shift_multi(lat, psi, s), 1)
    return _bc(lat.epsilon() * lat.eta5(), 1) * acc / 16.0


def sw_dslash(lat: Lattice, U, psi, mass, r=1.0, dagger=False, W16=None):
    """(D_SW + m) psi, or its adjoint.  Gamma55 from the literal symmetrised
    C-product unless the 16 hypercube transports W16 are given."""
    g55 = gamma55_literal(lat, U, psi) if W16 is None else gamma55_from_transport(lat, W16, psi)
    sgn = -1.0 if dagger else 1.0
    return sgn * staggered(lat, U, psi) + r * (psi - g55) + mass * psi


# ---------------------------------------------------------------- Wilson

_G, _G5 = gamma_matrices()


def _spin(g, psi):
    return np.einsum("st,...tb->...sb", g, psi)


def wilson_dslash(lat: Lattice, U, psi, mass, r=1.0, dagger=False):
    """(D_W + m) psi, or its adjoint (gamma_mu -> -gamma_mu)."""
    sg = -1.0 if dagger else 1.0
    out = (4.0 * r + mass) * psi
    for mu in range(4):
        f = hop_fwd(lat, U, psi, mu, nint=2)
        b = hop_bwd(lat, U, psi, mu, nint=2)
        out = out - 0.5 * (r * f - sg * _spin(_G[mu], f) + r * b + sg * _spin(_G[mu], b))
    return out


def apply_gamma5(psi):
    return _spin(_G5, psi)


# ---------------------------------------------------------------- gauge transforms


def gauge_transform_links(lat: Lattice, U, Omega):
    """U_mu(x) -> Omega(x) U_mu(x) Omega(x+mu)^+ (Omega in lattice shape (...,3,3))."""
    return [Omega @ U[mu] @ _dag(lat.shift_links(Omega, [1 if nu == mu else 0 for nu in range(4)]))
            for mu in range(4)]


def gauge_transform_field(Omega, psi, nint=1):
    return _mul(Omega, psi, nint)
