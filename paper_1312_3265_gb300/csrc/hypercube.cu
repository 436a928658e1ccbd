// Hypercube transports W(x,s) of the staggered Wilson term (Sec. 3: the 16
// hypercube neighbours of the "8+16" stencil): the average over the 24
// orderings of the 4-link path from x to x+s, for the 8 stored displacements
// s = (s0, s1, s2, +1).
//
// The sum over orderings is built by dynamic programming over the walked
// directions, forward from x: for a set S of directions with signs s_S,
//   F(S) = sum_{mu in S} F(S \ mu) L_mu(x + s_{S \ mu}),   F({mu}) = L_mu(x),
// with L_mu(y) = U_mu(y) for s_mu = +1 and U_mu(y - mu)^+ for s_mu = -1, and
// W(x,s) = F({0,1,2,3}) / 24.  F(S) depends only on the signs inside S, so the
// 8 displacements share it: 18 two-direction and 20 three-direction partial
// sums (the signs of directions 0-2 free, direction 3 always +1) and the 8
// full ones take 36 + 60 + 32 = 128 matrix products per site, against 8 x 28
// = 224 when each displacement is built on its own.
//
// Eight threads per site, in one warp: each builds some of the partial sums
// in shared memory, then thread k assembles W(x, s_k).  FP64 throughout.
#include "internal.h"
#include "common.cuh"

namespace swc {

namespace {

// The partial sums of a site: (direction mask S, sign bits on S), bit mu of
// the sign bits set when s_mu = -1; level 2 then level 3, masks increasing,
// sign patterns increasing.  pred: for each direction mu in S (increasing),
// the slot of F(S \ mu) among the level-2 sums (level 3) or the level-3 sums
// (the full sums, one per stored displacement k).
struct HcTables {
  unsigned char mask2[18], sg2[18];
  unsigned char mask3[20], sg3[20], mu3[20][3], pred3[20][3];
  unsigned char pred4[8][4];
};

constexpr int popc4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

constexpr HcTables make_hc_tables() {
  HcTables t{};
  int n2 = 0, n3 = 0;
  for (int S = 0; S < 16; ++S) {
    const int lv = popc4(S);
    if (lv != 2 && lv != 3) continue;
    const int free = S & 7;  // directions whose sign varies
    for (int sg = 0; sg < 8; ++sg) {
      if (sg & ~free) continue;
      if (lv == 2) {
        t.mask2[n2] = (unsigned char)S;
        t.sg2[n2] = (unsigned char)sg;
        ++n2;
      } else {
        t.mask3[n3] = (unsigned char)S;
        t.sg3[n3] = (unsigned char)sg;
        ++n3;
      }
    }
  }
  for (int j = 0; j < 20; ++j) {
    int q = 0;
    for (int mu = 0; mu < 4; ++mu) {
      if (!((t.mask3[j] >> mu) & 1)) continue;
      const int T = t.mask3[j] & ~(1 << mu), sg = t.sg3[j] & T;
      int slot = 0;
      for (int i = 0; i < 18; ++i)
        if (t.mask2[i] == T && t.sg2[i] == sg) slot = i;
      t.mu3[j][q] = (unsigned char)mu;
      t.pred3[j][q] = (unsigned char)slot;
      ++q;
    }
  }
  for (int k = 0; k < 8; ++k)
    for (int mu = 0; mu < 4; ++mu) {
      const int T = 15 & ~(1 << mu), sg = k & T;
      int slot = 0;
      for (int j = 0; j < 20; ++j)
        if (t.mask3[j] == T && t.sg3[j] == sg) slot = j;
      t.pred4[k][mu] = (unsigned char)slot;
    }
  return t;
}

__constant__ HcTables kHc = make_hc_tables();

constexpr int kHcSites = 8;  // sites per 64-thread block (8 threads per site)

}  // namespace

__global__ void __launch_bounds__(64) hypercube_kernel(Geom g, GaugeC64 U, double2* __restrict__ W) {
  __shared__ double2 part[kHcSites][38][9];  // level-2 sums in 0..17, level-3 sums in 18..37
  const int ls = threadIdx.x >> 3, t = threadIdx.x & 7;
  const int n = blockIdx.x * kHcSites + ls;
  const bool valid = n < g.V;
  int x[4] = {0, 0, 0, 0}, df[4] = {0, 0, 0, 0}, db[4] = {0, 0, 0, 0};
  if (valid) {
    coords(g, n, x);
    hop_deltas(g, n, x, df, db);
  }
  // L_mu(y) for sign bit neg; a hop along mu from y reads only x_mu, which the
  // walked directions (never mu itself) leave unchanged, so db[mu] applies at y
  auto link = [&](int mu, int neg, int y) -> M3<double> {
    return neg ? dag(U.link(y + db[mu], mu)) : U.link(y, mu);
  };
  // x + s_T for the directions in T with the signs sg
  auto pos = [&](int T, int sg) {
    int y = n;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
      if ((T >> mu) & 1) y += ((sg >> mu) & 1) ? db[mu] : df[mu];
    return y;
  };
  auto store = [&](int slot, const M3<double>& M) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) part[ls][slot][i * 3 + j] = make_double2(M.e[i][j].re, M.e[i][j].im);
  };
  auto load = [&](int slot) {
    M3<double> M;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 v = part[ls][slot][i * 3 + j];
        M.e[i][j] = {v.x, v.y};
      }
    return M;
  };
  if (valid) {
    // two directions a < b: F = L_a(x) L_b(x + s_a) + L_b(x) L_a(x + s_b)
    for (int i = t; i < 18; i += 8) {
      const int S = kHc.mask2[i], sg = kHc.sg2[i];
      const int a = __ffs(S) - 1, b = __ffs(S & ~(1 << a)) - 1;
      const int na = (sg >> a) & 1, nb = (sg >> b) & 1;
      M3<double> M = mm(link(a, na, n), link(b, nb, pos(1 << a, sg)));
      madd(M, mm(link(b, nb, n), link(a, na, pos(1 << b, sg))));
      store(i, M);
    }
  }
  __syncwarp();
  if (valid) {
    // three directions: F(S) = sum_mu F(S \ mu) L_mu(x + s_{S \ mu})
    for (int j = (t + 6) & 7; j < 20; j += 8) {
      const int S = kHc.mask3[j], sg = kHc.sg3[j];
      M3<double> M;
#pragma unroll 1
      for (int q = 0; q < 3; ++q) {
        const int mu = kHc.mu3[j][q];
        const M3<double> term = mm(load(kHc.pred3[j][q]), link(mu, (sg >> mu) & 1, pos(S & ~(1 << mu), sg)));
        if (q == 0) M = term; else madd(M, term);
      }
      store(18 + j, M);
    }
  }
  __syncwarp();
  if (valid) {
    // all four directions for displacement k = t
    const int k = t;
    M3<double> M;
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      const M3<double> term = mm(load(18 + kHc.pred4[k][mu]), link(mu, (k >> mu) & 1, pos(15 & ~(1 << mu), k)));
      if (mu == 0) M = term; else madd(M, term);
    }
    double2* out = W + ((size_t)n * 8 + k) * 9;
    const double w = 1.0 / 24.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) out[i * 3 + j] = make_double2(w * M.e[i][j].re, w * M.e[i][j].im);
  }
}

int hypercube_build_f64(const Geom& g, const double2* U, double2* W, cudaStream_t st) {
  const long long grid = ((long long)g.V + kHcSites - 1) / kHcSites;
  hypercube_kernel<<<(unsigned)grid, 64, 0, st>>>(g, GaugeC64{U}, W);
  note_launches(1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e);
}

}  // namespace swc
