"""The condition-number estimate reported with every solve: the extreme
eigenvalues of the Lanczos tridiagonal built from CG's (alpha, beta)
(csrc/ritz.h), compiled for the host and pinned on matrices of known
spectrum (no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ritz(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("ritz") / "ritz"
    subprocess.run([cxx, "-std=c++17", "-O2", os.path.join(HERE, "host", "ritz.cc"), "-o", str(exe)],
                   check=True, capture_output=True)

    def run(h):
        h = np.asarray(h, dtype=np.float64).reshape(-1, 2)
        text = f"{len(h)}\n" + "\n".join(f"{float(a):.17g} {float(b):.17g}" for a, b in h) + "\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, timeout=60, check=True)
        lo, hi = (float(v) for v in out.stdout.split())
        return lo, hi
    return run


def cg_coefficients(A, b, k):
    """(alpha_j, beta_j) of k iterations of textbook CG on A x = b, x0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    out = []
    for _ in range(k):
        Ap = A @ p
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        beta = rr_new / rr
        out.append((alpha, beta))
        p = r + beta * p
        rr = rr_new
    return np.array(out)


def spd(eigs, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((len(eigs), len(eigs))))
    return Q @ np.diag(eigs) @ Q.T, rng.standard_normal(len(eigs))


def test_full_run_recovers_the_extreme_eigenvalues(ritz):
    """n iterations on an n x n matrix: the Ritz values are A's eigenvalues, so
    the extremes are the spectrum's ends (here 1 and 40, 24 equally spaced)."""
    eigs = np.linspace(1.0, 40.0, 24)
    A, b = spd(eigs, 1)
    lo, hi = ritz(cg_coefficients(A, b, 24))
    assert lo == pytest.approx(1.0, rel=1e-8) and hi == pytest.approx(40.0, rel=1e-8)


def test_ritz_extremes_move_outward_inside_the_spectrum(ritz):
    """Cauchy interlacing: the leading k x k tridiagonals' extreme eigenvalues
    never leave [lambda_min(A), lambda_max(A)], lambda_min(T_k) never grows and
    lambda_max(T_k) never shrinks with k."""
    eigs = np.geomspace(0.5, 300.0, 60)
    A, b = spd(eigs, 2)
    h = cg_coefficients(A, b, 30)
    prev_lo, prev_hi = np.inf, -np.inf
    for k in range(1, 31):
        lo, hi = ritz(h[:k])
        assert 0.5 * (1 - 1e-9) <= lo <= hi <= 300.0 * (1 + 1e-9)
        assert lo <= prev_lo * (1 + 1e-12) and hi >= prev_hi * (1 - 1e-12)
        prev_lo, prev_hi = lo, hi
    assert hi == pytest.approx(300.0, rel=1e-3)  # the top converges first (well separated)


def test_one_iteration_is_the_rayleigh_quotient(ritz):
    """T_1 = [1/alpha_0] and 1/alpha_0 = b.A b / b.b (the Rayleigh quotient of b)."""
    A, b = spd(np.linspace(2.0, 9.0, 7), 3)
    lo, hi = ritz(cg_coefficients(A, b, 1))
    rq = (b @ A @ b) / (b @ b)
    assert lo == pytest.approx(rq, rel=1e-12) and hi == pytest.approx(rq, rel=1e-12)


def test_degenerate_inputs(ritz):
    assert ritz([]) == (0.0, 0.0)
    assert ritz([[-1.0, 0.5], [1.0, 0.2]]) == (0.0, 0.0)  # a non-positive alpha: no estimate
