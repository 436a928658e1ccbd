// Condition-number estimate from CG's own coefficients (host code only, so
// that the host tests can compile it without the kernels).
#pragma once
#include <cmath>
#include <vector>

namespace swc {

// Extreme eigenvalues of the k x k Lanczos tridiagonal built from CG's
// (alpha_j, beta_j) (Golub & Van Loan, Sec. 10.2): diagonal
// 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j.
// Its eigenvalues (Ritz values) lie inside the spectrum of A and the extremes
// converge first, so lambda_max/lambda_min estimates the condition number
// kappa of (D+m)^+(D+m) (Sec. 3) from below.  Sturm-sequence bisection.
inline void ritz_extremes(const double* h, int k, double* lmin, double* lmax) {
  *lmin = *lmax = 0.0;
  if (k < 1) return;
  std::vector<double> d(k), e2(k, 0.0);
  for (int j = 0; j < k; ++j) {
    const double a = h[2 * j];
    if (!(a > 0.0)) return;
    d[j] = 1.0 / a + (j > 0 ? h[2 * (j - 1) + 1] / h[2 * (j - 1)] : 0.0);
    if (j + 1 < k) e2[j] = h[2 * j + 1] / (a * a);
  }
  double lo = d[0], hi = d[0];
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? sqrt(e2[j - 1]) : 0.0) + (j + 1 < k ? sqrt(e2[j]) : 0.0);
    lo = fmin(lo, d[j] - r);
    hi = fmax(hi, d[j] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double q = 1.0;
    for (int j = 0; j < k; ++j) {
      q = d[j] - x - (j > 0 ? e2[j - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      c += (q < 0.0);
    }
    return c;
  };
  auto kth = [&](int want) {  // smallest x with count_below(x) >= want
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
      const double m = 0.5 * (a + b);
      if (count_below(m) >= want) b = m; else a = m;
    }
    return 0.5 * (a + b);
  };
  *lmin = kth(1);
  *lmax = kth(k);
}

}  // namespace swc
