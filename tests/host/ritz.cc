// Host check of the condition-number estimate (csrc/ritz.h): reads k and then
// k pairs (alpha_j, beta_j) of a CG run from stdin and prints the extreme Ritz
// values lambda_min, lambda_max.
#include <cstdio>
#include <vector>

#include "../../paper_1312_3265_gb300/csrc/ritz.h"

int main() {
  int k = 0;
  if (std::scanf("%d", &k) != 1 || k < 0) return 2;
  std::vector<double> h(2 * static_cast<size_t>(k) + 2, 0.0);
  for (int j = 0; j < 2 * k; ++j)
    if (std::scanf("%lf", &h[j]) != 1) return 2;
  double lo = 0.0, hi = 0.0;
  swc::ritz_extremes(h.data(), k, &lo, &hi);
  std::printf("%.17g %.17g\n", lo, hi);
  return 0;
}
