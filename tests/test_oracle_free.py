"""Oracle pins in the free field (U = 1): closed-form spectra and the paper's
8/sqrt(5) condition-number ratio (Sec. 3)."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import Lattice, operators as ops, dense
from conftest import unit_links

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def free(dims):
    lat = Lattice(dims)
    return lat, lat.links(unit_links(lat.volume))


def reduced_momenta(dims):
    """Reduced Brillouin zone of the staggered field: p_mu = 2 pi n / L_mu in [0, pi)."""
    axes = [[2 * np.pi * n / L for n in range(L // 2)] for L in dims]
    return list(itertools.product(*axes))


def sw_free_eigs(dims, m, r):
    """Closed form: per reduced momentum p, 16 modes m + r(1 - sig c) + i tau s with
    c = prod |cos p|, s = sqrt(sum sin^2 p), sig, tau = +-1, each 4-fold; x3 colours."""
    out = []
    for p in reduced_momenta(dims):
        c = np.prod(np.abs(np.cos(p)))
        s = np.sqrt(np.sum(np.sin(p) ** 2))
        for sig in (1, -1):
            for tau in (1, -1):
                out += [m + r * (1 - sig * c) + 1j * tau * s] * 4 * 3
    return np.array(out)


def wilson_free_eigs(dims, m, r):
    """Closed form: m + r sum(1 - cos p) +- i sqrt(sum sin^2 p), each 2-fold per
    momentum p = 2 pi n / L, x3 colours."""
    out = []
    axes = [[2 * np.pi * n / L for n in range(L)] for L in dims]
    for p in itertools.product(*axes):
        re = m + r * np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(np.array(p)) ** 2))
        out += [re + 1j * im, re - 1j * im] * 2 * 3
    return np.array(out)


def same_multiset(a, b, tol):
    key = lambda z: (np.round(z.real, 6), np.round(z.imag, 6))
    a = sorted(a, key=key)
    b = sorted(b, key=key)
    return len(a) == len(b) and np.max(np.abs(np.array(a) - np.array(b))) < tol


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 2, 6, 2)])
def test_sw_free_spectrum(dims):
    lat, U = free(dims)
    m, r = 0.1, 1.0
    ev = np.linalg.eigvals(dense.sw_matrix(lat, U, m, r))
    assert same_multiset(ev, sw_free_eigs(dims, m, r), 1e-9)


@pytest.mark.parametrize("r", [0.5, 1.75])
def test_free_spectra_at_other_wilson_parameters(r):
    """The closed forms hold for any r (the Wilson term of either operator
    scales with it, the hopping term does not)."""
    dims, m = (4, 2, 2, 2), 0.07
    lat, U = free(dims)
    assert same_multiset(np.linalg.eigvals(dense.sw_matrix(lat, U, m, r)), sw_free_eigs(dims, m, r), 1e-9)
    assert same_multiset(np.linalg.eigvals(dense.wilson_matrix(lat, U, m, r)), wilson_free_eigs(dims, m, r), 1e-9)


def test_sw_free_2x4_two_eigenvalues_and_two_flavours():
    lat, U = free((2, 2, 2, 2))
    m, r = 0.05, 1.0
    ev = np.linalg.eigvals(dense.sw_matrix(lat, U, m, r))
    assert np.sum(np.abs(ev - m) < 1e-12) == 24 and np.sum(np.abs(ev - (m + 2 * r)) < 1e-12) == 24
    # massless: 8 zero modes per colour = 2 of the 4 staggered tastes survive
    ev0 = np.linalg.eigvals(dense.sw_matrix(lat, U, 0.0, r))
    assert np.sum(np.abs(ev0) < 1e-12) == 8 * 3


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 2, 2)])
def test_wilson_free_spectrum(dims):
    lat, U = free(dims)
    m, r = 0.1, 1.0
    ev = np.linalg.eigvals(dense.wilson_matrix(lat, U, m, r))
    assert same_multiset(ev, wilson_free_eigs(dims, m, r), 1e-9)


def test_wilson_free_2x4_multiplicities():
    lat, U = free((2, 2, 2, 2))
    m, r = 0.05, 1.0
    ev = np.linalg.eigvals(dense.wilson_matrix(lat, U, m, r)).real
    counts = [int(np.sum(np.abs(ev - (m + 2 * r * k)) < 1e-12)) for k in range(5)]
    assert counts == [4 * 3, 16 * 3, 24 * 3, 16 * 3, 4 * 3]


def test_free_condition_numbers_and_paper_ratio():
    """kappa^(1/2) of (D+m)^+(D+m): SW sqrt(4 + (r+m)^2)/m, W (8r+m)/m on 4^4, whose
    ratio tends to 8/sqrt(5) ~ 3.58 as m -> 0 (Sec. 3)."""
    lat, U = free((4, 4, 4, 4))
    for m in (0.01, 0.2):
        ksw = dense.condition_number(dense.sw_matrix(lat, U, m))
        kw = dense.condition_number(dense.wilson_matrix(lat, U, m))
        assert abs(np.sqrt(ksw) - np.sqrt(4 + (1 + m) ** 2) / m) < 1e-7 * np.sqrt(ksw)
        assert abs(np.sqrt(kw) - (8 + m) / m) < 1e-6 * np.sqrt(kw)
    g = GOLDEN["free_field_sqrt_kappa_ratio_limit"]
    ratio = (8 + 1e-3) / np.sqrt(4 + (1 + 1e-3) ** 2)  # closed forms just checked
    assert round(ratio, g["digits_printed"]) == g["value"]
    assert abs(8 / np.sqrt(5) - g["value"]) < 0.005


def test_free_staggered_commutes_with_gamma55():
    lat, U = free((4, 4, 4, 4))
    v = np.random.default_rng(0).normal(size=lat.shape + (3,)) + 0j
    a = ops.staggered(lat, U, ops.gamma55_literal(lat, U, v))
    b = ops.gamma55_literal(lat, U, ops.staggered(lat, U, v))
    assert np.abs(a - b).max() < 1e-13


def test_free_gamma55_square():
    # 2^4: every momentum is a zone corner, Gamma55^2 = 1 exactly.
    lat, U = free((2, 2, 2, 2))
    v = np.random.default_rng(1).normal(size=lat.shape + (3,)) + 0j
    g = ops.gamma55_literal(lat, U, ops.gamma55_literal(lat, U, v))
    assert np.abs(g - v).max() < 1e-14
    # 4^4: Gamma55 has eigenvalues +- prod_mu |cos p_mu|, 8-fold per reduced momentum.
    lat, U = free((4, 4, 4, 4))
    G = dense.matrix(lambda x: ops.gamma55_literal(lat, U, x), lat, (3,))
    ev = np.sort(np.linalg.eigvalsh(G))
    want = []
    for p in reduced_momenta(lat.dims):
        c = np.prod(np.abs(np.cos(p)))
        want += [c] * 8 * 3 + [-c] * 8 * 3
    assert np.abs(ev - np.sort(want)).max() < 1e-12


def test_stencil_neighbour_counts():
    """Staggered Wilson couples a site to 8 + 16 others, Wilson to 8 with rank-2
    spin projectors at r = 1 (Sec. 3, after Eq. 4); random links so no entry
    cancels by accident."""
    import lattice_synth as ls
    g = GOLDEN["neighbours_per_site"]
    lat = Lattice((4, 4, 4, 4))
    U = lat.links(ls.su3_links(lat.dims, 3, 0.5))
    M = dense.sw_matrix(lat, U, 0.1).reshape(lat.volume, 3, lat.volume, 3)
    blocks = np.abs(M).max(axis=(1, 3)) > 1e-14
    assert np.all(blocks.sum(axis=1) == 1 + g["staggered_wilson"])
    Mw = dense.wilson_matrix(lat, U, 0.1).reshape(lat.volume, 12, lat.volume, 12)
    bw = np.abs(Mw).max(axis=(1, 3)) > 1e-14
    assert np.all(bw.sum(axis=1) == 1 + g["wilson"])
    G, _ = ops.gamma_matrices()
    for mu in range(4):
        assert np.linalg.matrix_rank(np.eye(4) - G[mu]) == g["wilson_spin_components_after_projection"]


def antiperiodic_momenta(dims, reduced):
    """Free-field momenta with the antiperiodic time boundary: p_mu = 2 pi n / L_mu
    for mu < 3, p_3 = (2n + 1) pi / L_3; n over the full zone, or over [0, pi)
    (the staggered reduced zone)."""
    axes = []
    for mu, L in enumerate(dims):
        ns = range(L // 2) if reduced else range(L)
        axes.append([((2 * n + 1) if mu == 3 else 2 * n) * np.pi / L for n in ns])
    return list(itertools.product(*axes))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (4, 2, 2, 6)])
def test_sw_free_spectrum_antiperiodic(dims):
    """The antiperiodic time boundary shifts p_3 by pi / L_3 and changes nothing
    else: the same closed form per reduced momentum (Gamma55's corner hops that
    cross the boundary carry its sign too)."""
    lat = Lattice(dims, antiperiodic_t=True)
    U = lat.links(unit_links(lat.volume))
    m, r = 0.1, 1.0
    want = []
    for p in antiperiodic_momenta(dims, reduced=True):
        c = np.prod(np.abs(np.cos(p)))
        s = np.sqrt(np.sum(np.sin(p) ** 2))
        for sig in (1, -1):
            for tau in (1, -1):
                want += [m + r * (1 - sig * c) + 1j * tau * s] * 4 * 3
    ev = np.linalg.eigvals(dense.sw_matrix(lat, U, m, r))
    assert same_multiset(ev, np.array(want), 1e-9)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 4, 4)])
def test_wilson_free_spectrum_antiperiodic(dims):
    lat = Lattice(dims, antiperiodic_t=True)
    U = lat.links(unit_links(lat.volume))
    m, r = 0.1, 1.0
    want = []
    for p in antiperiodic_momenta(dims, reduced=False):
        re = m + r * np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(np.array(p)) ** 2))
        want += [re + 1j * im, re - 1j * im] * 2 * 3
    ev = np.linalg.eigvals(dense.wilson_matrix(lat, U, m, r))
    assert same_multiset(ev, np.array(want), 1e-9)
