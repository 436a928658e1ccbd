"""Lattice geometry for the oracle: fields as arrays shaped (..., L3, L2, L1, L0, *internal).

Canonical flat site order n = x0 + L0*(x1 + L1*(x2 + L2*x3)) maps onto the
C-ordered 4-D shape (L3, L2, L1, L0), so direction mu lives on lattice axis
3 - mu.  Fermion boundary conditions: periodic in every direction, or
antiperiodic in time (x3) when `antiperiodic_t` is set; links are periodic.
"""
from __future__ import annotations

import itertools

import numpy as np


class Lattice:
    def __init__(self, dims, antiperiodic_t=False):
        self.dims = tuple(int(d) for d in dims)
        if len(self.dims) != 4 or any(d < 2 or d % 2 for d in self.dims):
            raise ValueError("lattice extents must be four even numbers >= 2")
        self.antiperiodic_t = bool(antiperiodic_t)
        self.shape = tuple(reversed(self.dims))  # (L3, L2, L1, L0)
        self.volume = int(np.prod(self.dims))
        grids = np.meshgrid(*[np.arange(L) for L in self.shape], indexing="ij")
        # x[mu] as arrays of lattice shape
        self.x = [grids[3 - mu] for mu in range(4)]

    # ---- phases (computed from coordinates, Sec. 2) ----
    def eta(self, mu):
        """Staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})."""
        s = sum((self.x[nu] for nu in range(mu)), np.zeros(self.shape, dtype=np.int64))
        return 1 - 2 * (s % 2)

    def epsilon(self):
        """eps(x) = (-1)^(x0+x1+x2+x3)."""
        return 1 - 2 * (sum(self.x) % 2)

    def eta5(self):
        """eta5(x) = (-1)^(x0+x2)."""
        return 1 - 2 * ((self.x[0] + self.x[2]) % 2)

    # ---- layouts ----
    def links(self, U_flat):
        """Canonical (V,4,3,3) -> list of 4 arrays (L3,L2,L1,L0,3,3)."""
        U = np.asarray(U_flat).reshape(self.shape + (4, 3, 3))
        return [np.ascontiguousarray(U[..., mu, :, :]) for mu in range(4)]

    def field(self, v_flat, internal):
        """Canonical (..., V, *internal) -> (..., L3, L2, L1, L0, *internal)."""
        v = np.asarray(v_flat)
        lead = v.shape[: v.ndim - 1 - len(internal)]
        return v.reshape(lead + self.shape + tuple(internal))

    def flat(self, v, internal):
        lead = v.shape[: v.ndim - 4 - len(internal)]
        return v.reshape(lead + (self.volume,) + tuple(internal))

    # ---- shifts ----
    def shift(self, psi, mu, step, nint):
        """phi(x) = psi(x + step*mu_hat), with the fermion boundary sign when
        the hop wraps around the time extent (antiperiodic case)."""
        ax = -(nint + 1 + mu)
        phi = np.roll(psi, -step, axis=ax)
        if self.antiperiodic_t and mu == 3:
            T = self.dims[3]
            idx = [slice(None)] * phi.ndim
            # sites whose neighbour x3 + step lies outside [0, T)
            idx[ax] = T - 1 if step > 0 else 0
            phi[tuple(idx)] *= -1
        return phi

    def shift_links(self, A, offset):
        """A(x + offset) for a link-valued array (L3,L2,L1,L0,3,3), periodic."""
        for mu in range(4):
            if offset[mu]:
                A = np.roll(A, -offset[mu], axis=-(3 + mu))
        return A


def hypercube_vectors(stored_only=False):
    """Hypercube displacements s in {+1,-1}^4.

    Stored order (the 8 with s3 = +1): index k, s_mu = -1 iff bit mu of k is
    set (mu = 0,1,2).  The full list continues with k = 8..15 for s3 = -1,
    using the same bit rule on mu = 0,1,2.
    """
    out = []
    for k in range(16):
        s = [(-1 if (k >> mu) & 1 else 1) for mu in range(3)]
        s.append(1 if k < 8 else -1)
        out.append(tuple(s))
    return out[:8] if stored_only else out


PERMUTATIONS = list(itertools.permutations(range(4)))
