// Hypercube transports W(x,s) of the staggered Wilson term (Sec. 3: the 16
// hypercube neighbours of the "8+16" stencil): the average over the 24
// orderings of the 4-link path from x to x+s.
//
// Instead of 24 separate path products (72 matrix products) the sum over
// orderings is built by dynamic programming over subsets: for the set R of
// directions still to be walked, starting from x + s_{R^c},
//   P_R = sum_{mu in R} L_mu(x + s_{R^c}) P_{R \ mu},   P_{} = 1,
// with L_mu(y) = U_mu(y) for s_mu = +1 and U_mu(y - mu)^+ for s_mu = -1.
// Then W(x,s) = P_{0123} / 24.  That is 28 products per (x, s).
// One thread per (site, stored displacement); FP64 throughout.
#include "internal.h"
#include "common.cuh"

namespace swc {

__constant__ int kMaskOrder[15] = {1, 2, 4, 8, 3, 5, 6, 9, 10, 12, 7, 11, 13, 14, 15};

__global__ void __launch_bounds__(64) hypercube_kernel(Geom g, GaugeC64 U, double2* __restrict__ W) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 8LL * g.V) return;
  const int n = (int)(idx >> 3), k = (int)(idx & 7);
  const int s[4] = {(k & 1) ? -1 : 1, (k & 2) ? -1 : 1, (k & 4) ? -1 : 1, 1};
  int x[4];
  coords(g, n, x);
  M3<double> P[16];
  for (int q = 0; q < 15; ++q) {
    const int R = kMaskOrder[q];
    int y = n;  // x + s_{R^c}; a hop along mu only looks at x[mu]
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
      if (!((R >> mu) & 1)) y = hop(g, y, x, mu, s[mu]);
    M3<double> acc;
    bool first = true;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      if (!((R >> mu) & 1)) continue;
      const M3<double> L = (s[mu] > 0) ? U.link(y, mu) : dag(U.link(hop(g, y, x, mu, -1), mu));
      const int rest = R & ~(1 << mu);
      const M3<double> term = rest ? mm(L, P[rest]) : L;
      if (first) { acc = term; first = false; } else { madd(acc, term); }
    }
    P[R] = acc;
  }
  double2* out = W + ((size_t)n * 8 + k) * 9;
  const double w = 1.0 / 24.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) out[i * 3 + j] = make_double2(w * P[15].e[i][j].re, w * P[15].e[i][j].im);
}

int hypercube_build_f64(const Geom& g, const double2* U, double2* W, cudaStream_t st) {
  const long long total = 8LL * g.V;
  const int block = 64;
  const long long grid = (total + block - 1) / block;
  hypercube_kernel<<<(unsigned)grid, block, 0, st>>>(g, GaugeC64{U}, W);
  note_launches(1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e);
}

}  // namespace swc
