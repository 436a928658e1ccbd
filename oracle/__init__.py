"""FP64 CPU oracle for the staggered Wilson / Wilson CGNE path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link anything here: only the tests, the smoke check of __graft_entry__ and the
CPU-baseline leg of bench.py use it.  It shares no code with the CUDA library
(paper_1312_3265_gb300); the only module both sides use is lattice_synth,
which makes seeded inputs and holds none of the method's arithmetic.

What it computes, and where the paper fixes it:
  * the 2-flavour staggered Wilson operator D_SW + m (Sec. 1-2; the paper omits
    the explicit form and refers to Adams, PLB 699 (2011) 394).  Reading used:
        D_SW = D_st + r (1 - Gamma55),  Gamma55 = eps eta5 (C0 C1 C2 C3)_sym,
        C_mu = (V_mu + V_mu^+)/2,  V_mu psi(x) = U_mu(x) psi(x+mu).
    This reading reproduces the paper's only closed-form number, the free-field
    ratio kappa_W^(1/2)/kappa_SW^(1/2) -> 8/sqrt(5) for m -> 0 (Sec. 3);
  * the usual Wilson operator D_W + m (the 1392 flop/site operator of Eq. 4);
  * unpreconditioned CG on the normal equations (D+m)^+(D+m) psi = (D+m)^+ chi
    (Eq. 2), following Shewchuk's textbook algorithm cited in Sec. 3;
  * dense matrices and their spectra / condition numbers kappa = lmax/lmin of
    (D+m)^+(D+m) (Sec. 3) for small lattices.

Pins (tests/test_oracle_*.py, run with -m "not gpu"): free-field closed-form
spectra of both operators, the 8/sqrt(5) ratio, hermiticity structure
(D_st anti-Hermitian, Gamma55 Hermitian, eps-hermiticity of D_SW,
gamma5-hermiticity of D_W), gauge covariance under random SU(3) transforms,
[D_st, Gamma55] = 0 and Gamma55^2 = 1 in the 2^4 free field, literal Gamma55
against the hypercube-transport form, and CG against dense LU solves and CG's
finite-termination property.  Interacting-field iteration counts against the
paper's figure are parity unpinned (the paper's ensemble is not available).
"""
from .lattice import Lattice  # noqa: F401
from . import operators, cg, dense, site  # noqa: F401
