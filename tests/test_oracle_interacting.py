"""Oracle pins on random SU(3) backgrounds: hermiticity structure, gauge
covariance, hypercube-transport form of Gamma55, one-site evaluators, and CG
against dense LU solves and CG's finite termination."""
import numpy as np
import pytest

import lattice_synth as ls
from oracle import Lattice, operators as ops, dense, site
from oracle.cg import cg, cgne, vdot
from oracle.lattice import hypercube_vectors
from conftest import unit_links

DIMS = [(4, 4, 4, 4), (2, 4, 2, 6)]


def rand_field(lat, internal, seed):
    g = np.random.default_rng(seed)
    shape = lat.shape + internal
    return g.normal(size=shape) + 1j * g.normal(size=shape)


def setup(dims, apbc=False, seed=11, eps=0.5):
    lat = Lattice(dims, antiperiodic_t=apbc)
    return lat, lat.links(ls.su3_links(dims, seed, eps))


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("apbc", [False, True])
def test_sw_hermiticity_structure(dims, apbc):
    lat, U = setup(dims, apbc)
    a, b = rand_field(lat, (3,), 1), rand_field(lat, (3,), 2)
    # D_st anti-Hermitian, Gamma55 Hermitian
    assert abs(vdot(a, ops.staggered(lat, U, b)) + vdot(ops.staggered(lat, U, a), b)) < 1e-11
    g = ops.gamma55_literal
    assert abs(vdot(a, g(lat, U, b)) - vdot(g(lat, U, a), b)) < 1e-11
    # the dagger flag is the true adjoint
    m = 0.07
    lhs = vdot(a, ops.sw_dslash(lat, U, b, m, 1.0))
    rhs = vdot(ops.sw_dslash(lat, U, a, m, 1.0, dagger=True), b)
    assert abs(lhs - rhs) < 1e-11
    # eps-hermiticity: eps D_SW eps = D_SW^+
    e = lat.epsilon()[..., None]
    assert np.abs(e * ops.sw_dslash(lat, U, e * b, m) - ops.sw_dslash(lat, U, b, m, dagger=True)).max() < 1e-13


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("apbc", [False, True])
def test_wilson_gamma5_hermiticity(dims, apbc):
    lat, U = setup(dims, apbc)
    a, b = rand_field(lat, (4, 3), 3), rand_field(lat, (4, 3), 4)
    for r in (1.0, 0.7):
        lhs = vdot(a, ops.wilson_dslash(lat, U, b, 0.1, r))
        rhs = vdot(ops.wilson_dslash(lat, U, a, 0.1, r, dagger=True), b)
        assert abs(lhs - rhs) < 1e-10
        g5 = ops.apply_gamma5
        assert np.abs(g5(ops.wilson_dslash(lat, U, g5(b), 0.1, r))
                      - ops.wilson_dslash(lat, U, b, 0.1, r, dagger=True)).max() < 1e-13


def test_gamma_algebra():
    G, G5 = ops.gamma_matrices()
    for mu in range(4):
        assert np.allclose(G[mu], G[mu].conj().T)
        for nu in range(4):
            assert np.allclose(G[mu] @ G[nu] + G[nu] @ G[mu], 2 * np.eye(4) * (mu == nu))
    assert np.allclose(G5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("apbc", [False, True])
def test_gauge_covariance(apbc):
    dims = (4, 2, 4, 4)
    lat, U = setup(dims, apbc)
    Om = lat.links(np.repeat(ls.haar_su3(dims, 9)[:, None], 4, axis=1))[0]
    Ug = ops.gauge_transform_links(lat, U, Om)
    psi = rand_field(lat, (3,), 5)
    lhs = ops.sw_dslash(lat, Ug, ops.gauge_transform_field(Om, psi), 0.1)
    rhs = ops.gauge_transform_field(Om, ops.sw_dslash(lat, U, psi, 0.1))
    assert np.abs(lhs - rhs).max() < 1e-12
    chi = rand_field(lat, (4, 3), 6)
    lhs = ops.wilson_dslash(lat, Ug, ops.gauge_transform_field(Om, chi, 2), 0.1)
    rhs = ops.gauge_transform_field(Om, ops.wilson_dslash(lat, U, chi, 0.1), 2)
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (2, 4, 6, 2)])
@pytest.mark.parametrize("apbc", [False, True])
def test_gamma55_transport_form_matches_literal(dims, apbc):
    lat, U = setup(dims, apbc)
    W16 = ops.hypercube_all(lat, U, stored_only=False)
    psi = rand_field(lat, (3,), 7)
    a = ops.gamma55_literal(lat, U, psi)
    b = ops.gamma55_from_transport(lat, W16, psi)
    assert np.abs(a - b).max() < 1e-13


def test_transport_reverse_is_adjoint():
    """W(x, s) = W(x+s, -s)^+: the 8 stored displacements determine the other 8."""
    lat, U = setup((4, 4, 2, 4))
    W16 = ops.hypercube_all(lat, U, stored_only=False)
    svs = hypercube_vectors(False)
    for k, s in enumerate(svs):
        k_rev = svs.index(tuple(-v for v in s))
        back = lat.shift_links(W16[k_rev], list(s))  # W(x+s, -s)
        assert np.abs(W16[k] - np.conj(np.swapaxes(back, -1, -2))).max() < 1e-14


def test_transport_free_field_is_identity():
    lat = Lattice((4, 4, 4, 4))
    U = lat.links(unit_links(lat.volume))
    for W in ops.hypercube_all(lat, U):
        assert np.abs(W - np.eye(3)).max() < 1e-15


@pytest.mark.parametrize("apbc", [False, True])
def test_site_evaluators_match_whole_field(apbc):
    dims = (4, 2, 4, 6)
    lat, U = setup(dims, apbc)
    Uf = ls.su3_links(dims, 11, 0.5)
    psi = rand_field(lat, (3,), 8)
    spn = rand_field(lat, (4, 3), 9)
    full_sw = lat.flat(ops.sw_dslash(lat, U, psi, 0.03, 0.9, dagger=True), (3,))
    full_w = lat.flat(ops.wilson_dslash(lat, U, spn, 0.03, 0.8), (4, 3))
    W8 = ops.hypercube_all(lat, U)
    for n in (0, 5, 37, lat.volume - 1):
        got = site.sw_dslash_site(Uf, lat.flat(psi, (3,)), dims, n, 0.03, 0.9, True, apbc)
        assert np.abs(got - full_sw[n]).max() < 1e-13
        got = site.wilson_dslash_site(Uf, lat.flat(spn, (4, 3)), dims, n, 0.03, 0.8, False, apbc)
        assert np.abs(got - full_w[n]).max() < 1e-13
        for k, s in enumerate(hypercube_vectors(True)):
            assert np.abs(site.hypercube_site(Uf, dims, n, s) - lat.flat(W8[k], (3, 3))[n]).max() < 1e-14


@pytest.mark.parametrize("op", ["sw", "w"])
def test_cgne_matches_dense_lu(op):
    dims = (2, 2, 2, 4)
    lat, U = setup(dims, True, eps=0.3)
    m = 0.05
    if op == "sw":
        internal = (3,)
        D = lambda v: ops.sw_dslash(lat, U, v, m)
        Dd = lambda v: ops.sw_dslash(lat, U, v, m, dagger=True)
        M = dense.sw_matrix(lat, U, m)
    else:
        internal = (4, 3)
        D = lambda v: ops.wilson_dslash(lat, U, v, m)
        Dd = lambda v: ops.wilson_dslash(lat, U, v, m, dagger=True)
        M = dense.wilson_matrix(lat, U, m)
    chi = lat.field(ls.point_source(dims, int(np.prod(internal)), 1).reshape((-1,) + internal), internal)
    x, info = cgne(D, Dd, chi, 1e-12, 5000)
    x_lu = dense.direct_solve(M, chi.reshape(-1))
    kappa = dense.condition_number(M)
    err = np.linalg.norm(x.reshape(-1) - x_lu) / np.linalg.norm(x_lu)
    assert info["true_rel_resid"] < 1e-11
    assert err < kappa * 1e-12
    # the CG residual history decreases to tol and the count is finite
    assert info["history"][-1] <= 1e-12 and info["iters"] > 1


def test_cg_finite_termination_free_field():
    """CG on a matrix with k distinct eigenvalues ends in at most k steps: SW on
    the free 2^4 lattice has 2 ({m^2, (m+2r)^2}), Wilson 5 ((m+2rk)^2, k=0..4)."""
    lat = Lattice((2, 2, 2, 2))
    U = lat.links(unit_links(lat.volume))
    m = 0.1
    chi = rand_field(lat, (3,), 10)
    _, info = cgne(lambda v: ops.sw_dslash(lat, U, v, m),
                   lambda v: ops.sw_dslash(lat, U, v, m, dagger=True), chi, 1e-12, 50)
    assert info["iters"] <= 2
    # Wilson: exactly 5 steps already reach the solution up to rounding (kappa = 6561)
    chi = rand_field(lat, (4, 3), 11)
    _, info = cgne(lambda v: ops.wilson_dslash(lat, U, v, m),
                   lambda v: ops.wilson_dslash(lat, U, v, m, dagger=True), chi, 0.0, 5)
    assert info["true_rel_resid"] < 1e-10 and info["history"][4] > 1e-6


def test_cg_a_norm_error_decreases():
    """CG minimises the A-norm error over growing Krylov spaces, so it never increases."""
    g = np.random.default_rng(3)
    B = g.normal(size=(40, 40))
    A = B @ B.T + 0.1 * np.eye(40)
    b = g.normal(size=40)
    xs = np.linalg.solve(A, b)
    errs = []
    for k in range(1, 30):
        x, _ = cg(lambda v: A @ v, b, 0.0, k)
        e = x - xs
        errs.append(e @ A @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_transport_of_a_pure_gauge_is_path_independent(dims):
    """Pure-gauge links U_mu(x) = Omega(x) Omega(x+mu)^+: every path from x to
    x+s gives Omega(x) Omega(x+s)^+, so the average over the 24 orderings is
    exactly that for all 16 displacements (pins the order of the path
    products and the backward links U_mu(y-mu)^+)."""
    lat = Lattice(dims)
    Om = lat.links(np.repeat(ls.haar_su3(dims, 21)[:, None], 4, axis=1))[0]
    U = ops.gauge_transform_links(lat, lat.links(unit_links(lat.volume)), Om)
    W16 = ops.hypercube_all(lat, U, stored_only=False)
    for k, s in enumerate(hypercube_vectors(False)):
        want = Om @ np.conj(np.swapaxes(lat.shift_links(Om, list(s)), -1, -2))
        assert np.abs(W16[k] - want).max() < 1e-13, s


@pytest.mark.parametrize("apbc", [False, True])
def test_wilson_even_odd_schur_reading(apbc):
    """The even-odd Schur reading of the Wilson operator (the basis of
    SW_OP_WILSON_EVEN_ODD), from the oracle's operator alone: hops join
    opposite parities only, so the even part of D (v_e, 0) is M v_e (M = 4r +
    m); psi_e from D^ psi_e = chi^_e (chi^_e = chi_e - D_eo chi_o / M, D^ = M -
    D_eo D_oe / M, dense solve) and psi_o = (chi_o - D_oe psi_e) / M solve
    D psi = chi; for any psi_e the defect of (psi_e, psi_o(psi_e)) is (chi^_e -
    D^ psi_e, 0), and |D^+(defect)|^2 = M^2 |t|^2 + |(D^+)_oe t|^2."""
    lat, U = setup((4, 2, 2, 4), apbc, seed=21)
    even = ((sum(lat.x) % 2) == 0)[..., None, None]
    for r in (1.0, 0.7):
        m = 0.15
        M = 4 * r + m
        D = lambda v, dag=False: ops.wilson_dslash(lat, U, v, m, r, dagger=dag)
        ev = lambda v: np.where(even, v, 0)
        od = lambda v: np.where(even, 0, v)
        v = ev(rand_field(lat, (4, 3), 30))
        assert np.abs(ev(D(v)) - M * v).max() < 1e-13
        assert np.abs(ev(D(v, True)) - M * v).max() < 1e-13
        # D_eo u = even part of D (0, u_o); D_oe v = odd part of D (v_e, 0)
        Deo = lambda u: ev(D(od(u)))
        Doe = lambda w: od(D(ev(w)))
        Dhat = lambda w: M * ev(w) - Deo(Doe(w)) / M
        chi = rand_field(lat, (4, 3), 31)
        chih = ev(chi) - Deo(chi) / M
        # dense D^ on the even sites
        idx = np.flatnonzero(np.broadcast_to(even, lat.shape + (4, 3)).reshape(-1))
        n = idx.size
        A = np.zeros((n, n), dtype=complex)
        for k in range(n):
            e = np.zeros(lat.shape + (4, 3), dtype=complex).reshape(-1)
            e[idx[k]] = 1.0
            A[:, k] = Dhat(e.reshape(lat.shape + (4, 3))).reshape(-1)[idx]
        psie = np.zeros(lat.shape + (4, 3), dtype=complex).reshape(-1)
        psie[idx] = np.linalg.solve(A, chih.reshape(-1)[idx])
        psie = psie.reshape(lat.shape + (4, 3))
        psi = psie + (od(chi) - Doe(psie)) / M
        assert np.abs(D(psi) - chi).max() < 1e-11
        # defect of an arbitrary psi_e with its psi_o rebuilt
        w = ev(rand_field(lat, (4, 3), 32))
        psi = w + (od(chi) - Doe(w)) / M
        t = chih - Dhat(w)
        defect = chi - D(psi)
        assert np.abs(defect - t).max() < 1e-12
        lhs = np.vdot(D(defect, True), D(defect, True)).real
        rhs = M * M * np.vdot(t, t).real + np.vdot(od(D(t, True)), od(D(t, True))).real
        assert abs(lhs - rhs) <= 1e-12 * lhs
