// Per-site operator application for both Dirac operators, generic over the
// storage layout (accessors from common.cuh) and the arithmetic type.
//
// Staggered Wilson (Sec. 1-2; operator of Adams, PLB 699 (2011) 394):
//   (D_SW + m) psi(x) = sgn/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^+ psi(x-mu)]
//                       + (r + m) psi(x)
//                       - r eps(x) eta5(x) / 16 sum_{s in {+-1}^4} W(x,s) psi(x+s)
//   sgn = +1, or -1 for the adjoint (D_st anti-Hermitian, Gamma55 Hermitian).
//   The 16 hypercube corners use the 8 stored transports: W(x,s) for s3 = +1,
//   and W(x,s) = W(x+s,-s)^+ (stored at the corner site) for s3 = -1.
//
// Wilson (Eq. 4's 1392 flop/site operator):
//   (D_W + m) psi(x) = (4r+m) psi(x) - 1/2 sum_mu [(r - c g_mu) U_mu(x) psi(x+mu)
//                                                 + (r + c g_mu) U_mu(x-mu)^+ psi(x-mu)]
//   c = +1, or -1 for the adjoint.  At r = 1 the factors (1 -+ g_mu) have rank 2
//   and the hop is done on projected 2-spinors ("8x2" of Sec. 3); other r use
//   the full 4-spinor.  DeGrand-Rossi basis: g_mu = [[0, A_mu], [A_mu^+, 0]].
#pragma once
#include "common.cuh"

namespace swc {

// eps(x) eta5(x) = (-1)^(x1 + x3)
__device__ __forceinline__ bool eps_eta5_neg(const int x[4]) { return ((x[1] + x[3]) & 1) != 0; }

template <typename T> __device__ __forceinline__ void neg3(V3<T>& v) {
#pragma unroll
  for (int i = 0; i < 3; ++i) v.c[i] = T(-1) * v.c[i];
}

// Offsets of the two hypercube corners paired with stored transport k
// (s_k = (s0, s1, s2, +1), bit mu of k set: s_mu = -1): the corner x + s_k,
// and x - s_k, whose transport W(x - s_k, s_k) gives W(x, -s_k) = W(x - s_k, s_k)^+.
__host__ __device__ inline void corner_offsets(int k, const int df[4], const int db[4], int& of, int& ob) {
  of = ((k & 1) ? db[0] : df[0]) + ((k & 2) ? db[1] : df[1]) + ((k & 4) ? db[2] : df[2]) + df[3];
  ob = ((k & 1) ? df[0] : db[0]) + ((k & 2) ? df[1] : db[1]) + ((k & 4) ? df[2] : db[2]) + db[3];
}

// acc += M v, acc += M^+ v, acc -= M^+ v: the accumulation runs through the
// fused multiply-adds of the product, so no separate additions are needed
// (the one-system operator of the FP64 residuals, bound by the FP64 pipe).
template <typename T> __device__ __forceinline__ void mv_acc(V3<T>& acc, const M3<T>& M, const V3<T>& v) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      acc.c[i].re = fma(M.e[i][j].re, v.c[j].re, acc.c[i].re);
      acc.c[i].re = fma(-M.e[i][j].im, v.c[j].im, acc.c[i].re);
      acc.c[i].im = fma(M.e[i][j].re, v.c[j].im, acc.c[i].im);
      acc.c[i].im = fma(M.e[i][j].im, v.c[j].re, acc.c[i].im);
    }
}
template <typename T>
__device__ __forceinline__ void mdv_acc(V3<T>& acc, const M3<T>& M, const V3<T>& v, T sign) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T mr = sign * M.e[j][i].re, mi = sign * M.e[j][i].im;  // sign is +-1: exact
      acc.c[i].re = fma(mr, v.c[j].re, acc.c[i].re);
      acc.c[i].re = fma(mi, v.c[j].im, acc.c[i].re);
      acc.c[i].im = fma(mr, v.c[j].im, acc.c[i].im);
      acc.c[i].im = fma(-mi, v.c[j].re, acc.c[i].im);
    }
}

template <typename T, typename G, typename Wt, typename In>
__device__ __forceinline__ V3<T> sw_site(const Geom& g, int n, const G& U, const Wt& W, const In& in,
                                         T mass, T r, bool dagger) {
  int x[4], df[4], db[4];
  coords(g, n, x);
  hop_deltas(g, n, x, df, db);
  // st = sum_mu eta_mu [U_mu(x) psi(x+mu) - U_mu(x-mu)^+ psi(x-mu)]
  V3<T> st = zero3<T>();
  int par = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    V3<T> pf = ld3<In, T>(in, n + df[mu]), pb = ld3<In, T>(in, n + db[mu]);
    if (mu == 3) {
      if (bc_flip(g, x, +1)) neg3(pf);
      if (bc_flip(g, x, -1)) neg3(pb);
    }
    if (mu == 0) {  // eta_0 = +1
      mv_acc(st, U.link(n, mu), pf);
      mdv_acc(st, U.link(n + db[mu], mu), pb, T(-1));
    } else {
      V3<T> d = zero3<T>();
      mv_acc(d, U.link(n, mu), pf);
      mdv_acc(d, U.link(n + db[mu], mu), pb, T(-1));
      const T eta = (par & 1) ? T(-1) : T(1);
#pragma unroll
      for (int i = 0; i < 3; ++i) st.c[i] = st.c[i] + eta * d.c[i];
    }
    par += x[mu];
  }
  // h = sum over the 16 corners of W(x,s) psi(x+s)
  V3<T> h = zero3<T>();
  const bool fflip = bc_flip(g, x, +1), bflip = bc_flip(g, x, -1);
#pragma unroll 2
  for (int k = 0; k < 8; ++k) {
    int of, ob;
    corner_offsets(k, df, db, of, ob);
    V3<T> pf = ld3<In, T>(in, n + of), pb = ld3<In, T>(in, n + ob);
    if (fflip) neg3(pf);
    if (bflip) neg3(pb);
    mv_acc(h, W.mat(n, k), pf);
    mdv_acc(h, W.mat(n + ob, k), pb, T(1));
  }
  const T hs = (eps_eta5_neg(x) ? r : -r) * T(0.0625);
  const T ss = dagger ? T(-0.5) : T(0.5);
  const V3<T> self = ld3<In, T>(in, n);
  V3<T> o;
#pragma unroll
  for (int i = 0; i < 3; ++i) o.c[i] = ss * st.c[i] + (r + mass) * self.c[i] + hs * h.c[i];
  return o;
}

template <typename T> struct Sp { V3<T> s[4]; };

template <typename In, typename T> struct SpLoader {
  static __device__ __forceinline__ Sp<T> load(const In& in, int n) {
    Sp<T> p;
#pragma unroll
    for (int s = 0; s < 4; ++s) p.s[s] = ld3<In, T>(in, n, 3 * s);
    return p;
  }
};
// float4 planes: a spinor is 6 sixteen-byte loads from one base address
template <> struct SpLoader<VecP32q<12>, float> {
  static __device__ __forceinline__ Sp<float> load(const VecP32q<12>& in, int n) {
    Sp<float> p;
    const float4* b = in.p + pk(n, 6, 0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float4 v = __ldg(b + q * 16);
      const int c0 = 2 * q, c1 = 2 * q + 1;
      p.s[c0 / 3].c[c0 % 3] = {v.x, v.y};
      p.s[c1 / 3].c[c1 % 3] = {v.z, v.w};
    }
    return p;
  }
};
template <typename In, typename T> __device__ __forceinline__ Sp<T> ld_sp(const In& in, int n) {
  return SpLoader<In, T>::load(in, n);
}

// h = (psi_u - c A_mu psi_d): the two independent spin rows of (1 - c g_mu) psi
template <typename T>
__device__ __forceinline__ void wproject(int mu, T c, const Sp<T>& p, V3<T>& h0, V3<T>& h1) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const cx<T> a0 = p.s[0].c[i], a1 = p.s[1].c[i], a2 = p.s[2].c[i], a3 = p.s[3].c[i];
    switch (mu) {
      case 0: h0.c[i] = a0 - c * times_i(a3); h1.c[i] = a1 - c * times_i(a2); break;
      case 1: h0.c[i] = a0 + c * a3;          h1.c[i] = a1 - c * a2;          break;
      case 2: h0.c[i] = a0 - c * times_i(a2); h1.c[i] = a1 + c * times_i(a3); break;
      default: h0.c[i] = a0 - c * a2;         h1.c[i] = a1 - c * a3;          break;
    }
  }
}
// acc += (1 - c g_mu) reconstructed from the transported rows h0, h1
template <typename T>
__device__ __forceinline__ void wreconstruct(int mu, T c, const V3<T>& h0, const V3<T>& h1, Sp<T>& acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const cx<T> b0 = h0.c[i], b1 = h1.c[i];
    acc.s[0].c[i] = acc.s[0].c[i] + b0;
    acc.s[1].c[i] = acc.s[1].c[i] + b1;
    switch (mu) {
      case 0: acc.s[2].c[i] = acc.s[2].c[i] + c * times_i(b1); acc.s[3].c[i] = acc.s[3].c[i] + c * times_i(b0); break;
      case 1: acc.s[2].c[i] = acc.s[2].c[i] - c * b1;          acc.s[3].c[i] = acc.s[3].c[i] + c * b0;          break;
      case 2: acc.s[2].c[i] = acc.s[2].c[i] + c * times_i(b0); acc.s[3].c[i] = acc.s[3].c[i] - c * times_i(b1); break;
      default: acc.s[2].c[i] = acc.s[2].c[i] - c * b0;         acc.s[3].c[i] = acc.s[3].c[i] - c * b1;          break;
    }
  }
}
// acc += (r - c g_mu) f for a full transported 4-spinor f
template <typename T>
__device__ __forceinline__ void wgeneral(int mu, T c, T r, const Sp<T>& f, Sp<T>& acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const cx<T> f0 = f.s[0].c[i], f1 = f.s[1].c[i], f2 = f.s[2].c[i], f3 = f.s[3].c[i];
    cx<T> g0, g1, g2, g3;  // g_mu f
    switch (mu) {
      case 0: g0 = times_i(f3); g1 = times_i(f2); g2 = T(-1) * times_i(f1); g3 = T(-1) * times_i(f0); break;
      case 1: g0 = T(-1) * f3;  g1 = f2;          g2 = f1;                   g3 = T(-1) * f0;          break;
      case 2: g0 = times_i(f2); g1 = T(-1) * times_i(f3); g2 = T(-1) * times_i(f0); g3 = times_i(f1); break;
      default: g0 = f2;         g1 = f3;          g2 = f0;                   g3 = f1;                  break;
    }
    acc.s[0].c[i] = acc.s[0].c[i] + r * f0 - c * g0;
    acc.s[1].c[i] = acc.s[1].c[i] + r * f1 - c * g1;
    acc.s[2].c[i] = acc.s[2].c[i] + r * f2 - c * g2;
    acc.s[3].c[i] = acc.s[3].c[i] + r * f3 - c * g3;
  }
}

template <typename T, bool R1, typename G, typename In>
__device__ __forceinline__ Sp<T> wilson_site(const Geom& g, int n, const G& U, const In& in,
                                             T mass, T r, bool dagger) {
  int x[4], df[4], db[4];
  coords(g, n, x);
  hop_deltas(g, n, x, df, db);
  Sp<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s) acc.s[s] = zero3<T>();
  const T sg = dagger ? T(-1) : T(1);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = n + df[mu], nb = n + db[mu];
    T bf = T(1), bb = T(1);
    if (mu == 3) {
      if (bc_flip(g, x, +1)) bf = T(-1);
      if (bc_flip(g, x, -1)) bb = T(-1);
    }
    const M3<T> Uf = U.link(n, mu);
    const M3<T> Ub = U.link(nb, mu);
    if (R1) {
      V3<T> h0, h1;
      const Sp<T> pf = ld_sp<In, T>(in, nf);
      wproject(mu, sg, pf, h0, h1);
      V3<T> u0 = mv(Uf, h0), u1 = mv(Uf, h1);
      if (bf < T(0)) { neg3(u0); neg3(u1); }
      wreconstruct(mu, sg, u0, u1, acc);
      const Sp<T> pb = ld_sp<In, T>(in, nb);
      wproject(mu, -sg, pb, h0, h1);
      u0 = mdv(Ub, h0);
      u1 = mdv(Ub, h1);
      if (bb < T(0)) { neg3(u0); neg3(u1); }
      wreconstruct(mu, -sg, u0, u1, acc);
    } else {
      const Sp<T> pf = ld_sp<In, T>(in, nf), pb = ld_sp<In, T>(in, nb);
      Sp<T> f, b;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        f.s[s] = mv(Uf, pf.s[s]);
        b.s[s] = mdv(Ub, pb.s[s]);
        if (bf < T(0)) neg3(f.s[s]);
        if (bb < T(0)) neg3(b.s[s]);
      }
      wgeneral(mu, sg, r, f, acc);
      wgeneral(mu, -sg, r, b, acc);
    }
  }
  const Sp<T> self = ld_sp<In, T>(in, n);
  const T diag = T(4) * r + mass;
  Sp<T> o;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int i = 0; i < 3; ++i) o.s[s].c[i] = diag * self.s[s].c[i] - T(0.5) * acc.s[s].c[i];
  return o;
}

// ------------------------------------------------------------------ two-lane colour products (FP32)
// u = M h for two colour vectors at once, held in the two lanes of float2
// registers (real parts in one array, imaginary parts in the other): one
// two-lane FMA does the work of two scalar ones, with the matrix entries
// broadcast to both lanes.
// u = M h (DAG = false) or M^+ h (DAG = true)
template <bool DAG>
__device__ __forceinline__ void mv_pair(const M3<float>& M, const float2 hre[3], const float2 him[3], float2 ure[3],
                                        float2 uim[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const cx<float> m0 = DAG ? M.e[0][i] : M.e[i][0];
    const float s = DAG ? -1.f : 1.f;  // conj: the imaginary parts change sign
    ure[i] = fmul2(bc2(m0.re), hre[0]);
    ure[i] = ffma2(bc2(-s * m0.im), him[0], ure[i]);
    uim[i] = fmul2(bc2(m0.re), him[0]);
    uim[i] = ffma2(bc2(s * m0.im), hre[0], uim[i]);
#pragma unroll
    for (int j = 1; j < 3; ++j) {
      const cx<float> m = DAG ? M.e[j][i] : M.e[i][j];
      ure[i] = ffma2(bc2(m.re), hre[j], ure[i]);
      ure[i] = ffma2(bc2(-s * m.im), him[j], ure[i]);
      uim[i] = ffma2(bc2(m.re), him[j], uim[i]);
      uim[i] = ffma2(bc2(s * m.im), hre[j], uim[i]);
    }
  }
}

}  // namespace swc

// ------------------------------------------------------------------ multi-system forms
// The same operators applied to NS systems at once: each link / transport is
// loaded once and applied to the NS vectors, so the gauge data crosses the
// memory hierarchy once per site instead of once per system.  System s lives
// `stride` complex numbers after system s-1; bit s of `act` selects the
// systems to compute (others are neither loaded nor written).
namespace swc {

template <typename Vec> __device__ __forceinline__ Vec sys_at(Vec v, int s, size_t stride) {
  v.p += s * stride;
  return v;
}
// paired storage: s systems further on, the pair and the lane move together
template <int NC> __device__ __forceinline__ VecP32x2<NC> sys_at(VecP32x2<NC> v, int s, size_t stride) {
  const int t = v.lane + s;
  v.p += (size_t)(t >> 1) * 2 * stride;
  v.lane = t & 1;
  return v;
}

template <typename T> __device__ __forceinline__ void axpy3(V3<T>& acc, T a, const V3<T>& v) {
#pragma unroll
  for (int i = 0; i < 3; ++i) acc.c[i] = acc.c[i] + a * v.c[i];
}

template <typename T, int NS, typename G, typename Wt, typename In, typename GG>
__device__ __forceinline__ void sw_site_multi(const GG& g, int n, const G& U, const Wt& W, const In& in,
                                              size_t stride, unsigned act, const T* mass, T r, bool dagger,
                                              V3<T>* out) {
  int x[4], df[4], db[4];
  coords(g, n, x);
  hop_deltas(g, n, x, df, db);
  V3<T> acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) acc[s] = zero3<T>();
  const T half = dagger ? T(-0.5) : T(0.5);
  int par = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = n + df[mu], nb = n + db[mu];
    const T eta = (par & 1) ? -half : half;
    T cf = eta, cb = -eta;
    if (mu == 3) {
      if (bc_flip(g, x, +1)) cf = -cf;
      if (bc_flip(g, x, -1)) cb = -cb;
    }
    const M3<T> Uf = U.link(n, mu);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (act & (1u << s)) axpy3(acc[s], cf, mv(Uf, ld3<In, T>(sys_at(in, s, stride), nf)));
    const M3<T> Ub = U.link(nb, mu);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (act & (1u << s)) axpy3(acc[s], cb, mdv(Ub, ld3<In, T>(sys_at(in, s, stride), nb)));
    par += x[mu];
  }
  const T hs = (eps_eta5_neg(x) ? r : -r) * T(0.0625);
  const T hf = bc_flip(g, x, +1) ? -hs : hs, hb = bc_flip(g, x, -1) ? -hs : hs;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    int of, ob;
    corner_offsets(k, df, db, of, ob);
    const int yf = n + of, yb = n + ob;
    const M3<T> Wf = W.mat(n, k);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (act & (1u << s)) axpy3(acc[s], hf, mv(Wf, ld3<In, T>(sys_at(in, s, stride), yf)));
    const M3<T> Wb = W.mat(yb, k);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (act & (1u << s)) axpy3(acc[s], hb, mdv(Wb, ld3<In, T>(sys_at(in, s, stride), yb)));
  }
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (act & (1u << s)) {
      const V3<T> self = ld3<In, T>(sys_at(in, s, stride), n);
      axpy3(acc[s], r + mass[s], self);
      out[s] = acc[s];
    }
}

// The same operator for NS (even) FP32 systems with the systems of each pair
// in the two lanes of float2 registers: one two-lane FMA does the work of two
// scalar ones, with the link and transport entries broadcast to both lanes.
// The 16 hypercube corners accumulate unscaled (their coefficients
// eps eta5 r/16 are one value per site, up to the time-boundary sign), and
// are scaled once per direction sign.  A lane whose system is not computed
// reads its partner's vector (never memory outside the batch) and is dropped.
template <int NS, typename G, typename Wt, typename In, typename GG>
__device__ __forceinline__ void sw_site_multi_pair(const GG& g, int n, const G& U, const Wt& W, const In& in,
                                                   size_t stride, unsigned act, const float* mass, float r,
                                                   bool dagger, V3<float>* out) {
  static_assert(NS % 2 == 0, "pairs of systems");
  constexpr int NP = NS / 2;
  int x[4], df[4], db[4];
  coords(g, n, x);
  hop_deltas(g, n, x, df, db);
  In lane0[NP], lane1[NP];
  bool on[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const unsigned a = (act >> (2 * q)) & 3u;
    on[q] = a != 0;
    lane0[q] = sys_at(in, (a & 1u) ? 2 * q : 2 * q + 1, stride);
    lane1[q] = sys_at(in, (a & 2u) ? 2 * q + 1 : 2 * q, stride);
  }
  float2 are[NP][3], aim[NP][3];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int i = 0; i < 3; ++i) are[q][i] = aim[q][i] = make_float2(0.f, 0.f);
  // packed vector of pair q at site y: lanes (first, second system)
  auto ldp = [&](int q, int y, float2 vre[3], float2 vim[3]) {
    if constexpr (is_paired<In>::value) {  // the pair's storage holds the lanes already
      const In b = sys_at(in, 2 * q, stride);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float4 w = __ldg(b.p + pk(y, 3, j));
        vre[j] = make_float2(w.x, w.y);
        vim[j] = make_float2(w.z, w.w);
      }
    } else {
      const V3<float> a = ld3<In, float>(lane0[q], y), b = ld3<In, float>(lane1[q], y);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        vre[j] = make_float2(a.c[j].re, b.c[j].re);
        vim[j] = make_float2(a.c[j].im, b.c[j].im);
      }
    }
  };
  const float half = dagger ? -0.5f : 0.5f;
  int par = 0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = n + df[mu], nb = n + db[mu];
    const float eta = (par & 1) ? -half : half;
    float cf = eta, cb = -eta;
    if (mu == 3) {
      if (bc_flip(g, x, +1)) cf = -cf;
      if (bc_flip(g, x, -1)) cb = -cb;
    }
    float2 vre[3], vim[3], ure[3], uim[3];
    const M3<float> Uf = U.link(n, mu);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (!on[q]) continue;
      ldp(q, nf, vre, vim);
      mv_pair<false>(Uf, vre, vim, ure, uim);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        are[q][i] = ffma2(bc2(cf), ure[i], are[q][i]);
        aim[q][i] = ffma2(bc2(cf), uim[i], aim[q][i]);
      }
    }
    const M3<float> Ub = U.link(nb, mu);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      if (!on[q]) continue;
      ldp(q, nb, vre, vim);
      mv_pair<true>(Ub, vre, vim, ure, uim);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        are[q][i] = ffma2(bc2(cb), ure[i], are[q][i]);
        aim[q][i] = ffma2(bc2(cb), uim[i], aim[q][i]);
      }
    }
    par += x[mu];
  }
  const float hs = (eps_eta5_neg(x) ? r : -r) * 0.0625f;
  const float hf = bc_flip(g, x, +1) ? -hs : hs, hb = bc_flip(g, x, -1) ? -hs : hs;
  // the 8 corners x + s (s3 = +1) by the stored W(x, s), then the 8 corners
  // x - s by W(x - s, s)^+
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    float2 hre[NP][3], him[NP][3];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int i = 0; i < 3; ++i) hre[q][i] = him[q][i] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      int of, ob;
      corner_offsets(k, df, db, of, ob);
      const int y = n + (side ? ob : of);
      const M3<float> M = side ? W.mat(y, k) : W.mat(n, k);
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        if (!on[q]) continue;
        float2 vre[3], vim[3];
        ldp(q, y, vre, vim);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const cx<float> m = side ? M.e[j][i] : M.e[i][j];
            const float mi = side ? -m.im : m.im;  // W^+: conjugate transpose
            hre[q][i] = ffma2(bc2(m.re), vre[j], hre[q][i]);
            hre[q][i] = ffma2(bc2(-mi), vim[j], hre[q][i]);
            him[q][i] = ffma2(bc2(m.re), vim[j], him[q][i]);
            him[q][i] = ffma2(bc2(mi), vre[j], him[q][i]);
          }
      }
    }
    const float c = side ? hb : hf;
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        are[q][i] = ffma2(bc2(c), hre[q][i], are[q][i]);
        aim[q][i] = ffma2(bc2(c), him[q][i], aim[q][i]);
      }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    if (!on[q]) continue;
    float2 vre[3], vim[3];
    ldp(q, n, vre, vim);
    const float2 d = make_float2(r + mass[2 * q], r + mass[2 * q + 1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      are[q][i] = ffma2(d, vre[i], are[q][i]);
      aim[q][i] = ffma2(d, vim[i], aim[q][i]);
      out[2 * q].c[i] = {are[q][i].x, aim[q][i].x};
      out[2 * q + 1].c[i] = {are[q][i].y, aim[q][i].y};
    }
  }
}

// ---- lean form of the spin-projected FP32 Wilson site (one system per thread)
// The same arithmetic as wilson_site_multi at r = 1, in an order that keeps
// fewer values live: each projected row h0, h1 is formed from the two spins
// it needs (the float4 units that hold them; a unit's other half is kept for
// the second row), and the transported rows are formed one colour at a time,
// from one row (or column) of the link, and reconstructed into the
// accumulator at once.
__device__ __forceinline__ cx<float> lo2(float4 v) { return {v.x, v.y}; }
__device__ __forceinline__ cx<float> hi2(float4 v) { return {v.z, v.w}; }

template <int MU>
__device__ __forceinline__ void wproject_rows(const float4* b, float c, V3<float>& h0, V3<float>& h1) {
  // component k = 3 spin + colour sits in unit k/2, half k%2
  if constexpr (MU < 2) {  // rows from spins (0, 3) and (1, 2)
    const float4 u0 = __ldg(b), u1 = __ldg(b + 16), u4 = __ldg(b + 64), u5 = __ldg(b + 80);
    const cx<float> s0[3] = {lo2(u0), hi2(u0), lo2(u1)}, s3[3] = {hi2(u4), lo2(u5), hi2(u5)};
#pragma unroll
    for (int i = 0; i < 3; ++i) h0.c[i] = MU == 0 ? s0[i] - c * times_i(s3[i]) : s0[i] + c * s3[i];
    const cx<float> c3 = hi2(u1), c8 = lo2(u4);
    const float4 u2 = __ldg(b + 32), u3 = __ldg(b + 48);
    const cx<float> s1[3] = {c3, lo2(u2), hi2(u2)}, s2[3] = {lo2(u3), hi2(u3), c8};
#pragma unroll
    for (int i = 0; i < 3; ++i) h1.c[i] = MU == 0 ? s1[i] - c * times_i(s2[i]) : s1[i] - c * s2[i];
  } else {  // rows from spins (0, 2) and (1, 3)
    const float4 u0 = __ldg(b), u1 = __ldg(b + 16), u3 = __ldg(b + 48), u4 = __ldg(b + 64);
    const cx<float> s0[3] = {lo2(u0), hi2(u0), lo2(u1)}, s2[3] = {lo2(u3), hi2(u3), lo2(u4)};
#pragma unroll
    for (int i = 0; i < 3; ++i) h0.c[i] = MU == 2 ? s0[i] - c * times_i(s2[i]) : s0[i] - c * s2[i];
    const cx<float> c3 = hi2(u1), c9 = hi2(u4);
    const float4 u2 = __ldg(b + 32), u5 = __ldg(b + 80);
    const cx<float> s1[3] = {c3, lo2(u2), hi2(u2)}, s3[3] = {c9, lo2(u5), hi2(u5)};
#pragma unroll
    for (int i = 0; i < 3; ++i) h1.c[i] = MU == 2 ? s1[i] + c * times_i(s3[i]) : s1[i] - c * s3[i];
  }
}

// acc += (1 - c g_mu) reconstructed from row i of the transported rows: one
// link row (fwd) or column (bwd, the adjoint) at a time
template <int MU, bool BWD>
__device__ __forceinline__ void whop_rows(const float2* q, float c, bool flip, const V3<float>& h0,
                                          const V3<float>& h1, Sp<float>& acc) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cx<float> m[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2 e = __ldg(q + (BWD ? (j * 3 + i) : (i * 3 + j)) * 16);
      m[j] = {e.x, e.y};
    }
    float r0, i0, r1, i1;
    if constexpr (!BWD) {  // the products of mv
      r0 = m[0].re * h0.c[0].re, i0 = m[0].re * h0.c[0].im;
      r0 = fma(-m[0].im, h0.c[0].im, r0);
      i0 = fma(m[0].im, h0.c[0].re, i0);
      cmac(r0, i0, m[1], h0.c[1]);
      cmac(r0, i0, m[2], h0.c[2]);
      r1 = m[0].re * h1.c[0].re, i1 = m[0].re * h1.c[0].im;
      r1 = fma(-m[0].im, h1.c[0].im, r1);
      i1 = fma(m[0].im, h1.c[0].re, i1);
      cmac(r1, i1, m[1], h1.c[1]);
      cmac(r1, i1, m[2], h1.c[2]);
    } else {  // the products of mdv
      r0 = m[0].re * h0.c[0].re, i0 = m[0].re * h0.c[0].im;
      r0 = fma(m[0].im, h0.c[0].im, r0);
      i0 = fma(-m[0].im, h0.c[0].re, i0);
      cjmac(r0, i0, m[1], h0.c[1]);
      cjmac(r0, i0, m[2], h0.c[2]);
      r1 = m[0].re * h1.c[0].re, i1 = m[0].re * h1.c[0].im;
      r1 = fma(m[0].im, h1.c[0].im, r1);
      i1 = fma(-m[0].im, h1.c[0].re, i1);
      cjmac(r1, i1, m[1], h1.c[1]);
      cjmac(r1, i1, m[2], h1.c[2]);
    }
    cx<float> b0 = {r0, i0}, b1 = {r1, i1};
    if (flip) {
      b0 = {-b0.re, -b0.im};
      b1 = {-b1.re, -b1.im};
    }
    acc.s[0].c[i] = acc.s[0].c[i] + b0;
    acc.s[1].c[i] = acc.s[1].c[i] + b1;
    if constexpr (MU == 0) {
      acc.s[2].c[i] = acc.s[2].c[i] + c * times_i(b1);
      acc.s[3].c[i] = acc.s[3].c[i] + c * times_i(b0);
    } else if constexpr (MU == 1) {
      acc.s[2].c[i] = acc.s[2].c[i] - c * b1;
      acc.s[3].c[i] = acc.s[3].c[i] + c * b0;
    } else if constexpr (MU == 2) {
      acc.s[2].c[i] = acc.s[2].c[i] + c * times_i(b0);
      acc.s[3].c[i] = acc.s[3].c[i] - c * times_i(b1);
    } else {
      acc.s[2].c[i] = acc.s[2].c[i] - c * b0;
      acc.s[3].c[i] = acc.s[3].c[i] - c * b1;
    }
  }
}

template <int MU, typename GG>
__device__ __forceinline__ void whop_lean(const GG& g, int n, const int x[4], const GaugeP32& U,
                                          const VecP32q<12>& in, float sg, Sp<float>& acc) {
  const int nf = hop(g, n, x, MU, +1), nb = hop(g, n, x, MU, -1);
  V3<float> h0, h1;
  wproject_rows<MU>(in.p + pk(nf, 6, 0), sg, h0, h1);
  whop_rows<MU, false>(U.p + pk(n, 36, MU * 9), sg, MU == 3 && bc_flip(g, x, +1), h0, h1, acc);
  wproject_rows<MU>(in.p + pk(nb, 6, 0), -sg, h0, h1);
  whop_rows<MU, true>(U.p + pk(nb, 36, MU * 9), -sg, MU == 3 && bc_flip(g, x, -1), h0, h1, acc);
}

template <typename GG>
__device__ __forceinline__ void wilson_site_lean(const GG& g, int n, const GaugeP32& U, const VecP32q<12>& in,
                                                 float mass, bool dagger, Sp<float>& out) {
  int x[4];
  coords(g, n, x);
  Sp<float> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s) acc.s[s] = zero3<float>();
  const float sg = dagger ? -1.f : 1.f;
  whop_lean<0>(g, n, x, U, in, sg, acc);
  whop_lean<1>(g, n, x, U, in, sg, acc);
  whop_lean<2>(g, n, x, U, in, sg, acc);
  whop_lean<3>(g, n, x, U, in, sg, acc);
  const Sp<float> self = ld_sp<VecP32q<12>, float>(in, n);
  const float diag = 4.f + mass;  // 4r + m at r = 1
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) out.s[k].c[i] = diag * self.s[k].c[i] - 0.5f * acc.s[k].c[i];
}

template <typename T, bool R1, int NS, typename G, typename In, typename GG>
__device__ __forceinline__ void wilson_site_multi(const GG& g, int n, const G& U, const In& in, size_t stride,
                                                  unsigned act, const T* mass, T r, bool dagger, Sp<T>* out) {
  // (neighbours computed where used: holding eight offsets costs the
  // register-capped Wilson kernels more than the few integer operations)
  int x[4];
  coords(g, n, x);
  Sp<T> acc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[s].s[k] = zero3<T>();
  const T sg = dagger ? T(-1) : T(1);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = hop(g, n, x, mu, +1), nb = hop(g, n, x, mu, -1);
    const bool ff = (mu == 3) && bc_flip(g, x, +1), fb = (mu == 3) && bc_flip(g, x, -1);
    const M3<T> Uf = U.link(n, mu);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (!(act & (1u << s))) continue;
      const Sp<T> p = ld_sp<In, T>(sys_at(in, s, stride), nf);
      if (R1) {
        V3<T> h0, h1;
        wproject(mu, sg, p, h0, h1);
        V3<T> u0 = mv(Uf, h0), u1 = mv(Uf, h1);
        if (ff) { neg3(u0); neg3(u1); }
        wreconstruct(mu, sg, u0, u1, acc[s]);
      } else {
        Sp<T> f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          f.s[k] = mv(Uf, p.s[k]);
          if (ff) neg3(f.s[k]);
        }
        wgeneral(mu, sg, r, f, acc[s]);
      }
    }
    const M3<T> Ub = U.link(nb, mu);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (!(act & (1u << s))) continue;
      const Sp<T> p = ld_sp<In, T>(sys_at(in, s, stride), nb);
      if (R1) {
        V3<T> h0, h1;
        wproject(mu, -sg, p, h0, h1);
        V3<T> u0 = mdv(Ub, h0), u1 = mdv(Ub, h1);
        if (fb) { neg3(u0); neg3(u1); }
        wreconstruct(mu, -sg, u0, u1, acc[s]);
      } else {
        Sp<T> f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          f.s[k] = mdv(Ub, p.s[k]);
          if (fb) neg3(f.s[k]);
        }
        wgeneral(mu, -sg, r, f, acc[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (!(act & (1u << s))) continue;
    const Sp<T> self = ld_sp<In, T>(sys_at(in, s, stride), n);
    const T diag = T(4) * r + mass[s];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) out[s].s[k].c[i] = diag * self.s[k].c[i] - T(0.5) * acc[s].s[k].c[i];
  }
}

}  // namespace swc
