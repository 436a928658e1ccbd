"""Unpreconditioned CG on the normal equations (Eq. 2), textbook form.

Solves A x = b with A = (D+m)^+(D+m) and b = (D+m)^+ chi, starting from x0
(zero unless given), following the conjugate-gradient algorithm of
Shewchuk's tutorial cited in Sec. 3:
    r0 = b - A x0,  p0 = r0
    alpha_k = |r_k|^2 / <p_k, A p_k>
    x_{k+1} = x_k + alpha_k p_k,   r_{k+1} = r_k - alpha_k A p_k
    beta_k  = |r_{k+1}|^2 / |r_k|^2,   p_{k+1} = r_{k+1} + beta_k p_k
stopping when |r_k| / |b| <= tol (the residual epsilon of Sec. 3).  The true
residual |b - A x| / |b| is recomputed at the end.
"""
from __future__ import annotations

import numpy as np


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_A, b, tol, max_iter, x0=None):
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    bnorm = np.sqrt(vdot(b, b).real)
    hist = [np.sqrt(rr) / bnorm]
    k = 0
    while hist[-1] > tol and k < max_iter:
        Ap = apply_A(p)
        alpha = rr / vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = vdot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
        hist.append(np.sqrt(rr) / bnorm)
    true = np.sqrt(vdot(b - apply_A(x), b - apply_A(x)).real) / bnorm
    return x, {"iters": k, "history": hist, "true_rel_resid": true}


def cgne(apply_D, apply_Ddag, chi, tol, max_iter, x0=None):
    """CG on (D+m)^+(D+m) psi = (D+m)^+ chi; apply_D / apply_Ddag include m."""
    b = apply_Ddag(chi)
    x, info = cg(lambda v: apply_Ddag(apply_D(v)), b, tol, max_iter, x0)
    info["b"] = b
    return x, info
