// Even-odd (Schur complement) preconditioned CGNE for the Wilson operator.
//
// The Wilson operator couples a site only to itself and to its nearest
// neighbours, which have the other parity (x0+x1+x2+x3 even or odd), so with
// the sites ordered even then odd
//   D + m = [[M, D_eo], [D_oe, M]],   M = 4r + m,
// D_eo, D_oe the hopping term between the parities.  The even-site Schur
// complement  D^ = M - D_eo D_oe / M  gives
//   chi^_e = chi_e - D_eo chi_o / M,   D^ psi_e = chi^_e,
//   psi_o  = (chi_o - D_oe psi_e) / M,
// and CGNE runs on D^+ D^ psi_e = D^+ chi^_e over the even half of the
// lattice.  (D^)^+ = M - (D^+)_eo (D^+)_oe / M has the same form with the
// adjoint hops.  This is the textbook preconditioning of the Wilson
// operator; the paper's cost comparison runs unpreconditioned CGNE, and the
// staggered Wilson operator has no such Schur form: its Gamma55 term hops by
// one step in every direction, so it couples sites of equal parity and its
// even-even block is not diagonal.
//
// Half-lattice fields: the sites of one parity in the order of their full
// index n (x0 fastest); the half index is h = n >> 1 (every extent is even, so
// each pair (2h, 2h+1) holds one site of each parity).  Every half-lattice
// vector of the solve is followed, per system, by a second half-lattice field
// of scratch: a D^ application first writes u = D_oe p into the scratch of p
// (a pre-pass over the odd sites), then computes M p - D_eo u / M on the even
// sites, reading u at the odd neighbours.
//
// The engine runs on a one-dimensional layout geometry of V/2 sites (the
// packed inner-precision fields are then in half-index order); the operators
// carry the full lattice geometry for their neighbours.  Convergence is
// decided on the full system: every FP64 reliable update of the Schur solve
// also yields the full system's normal-equation residual |b - A psi| / |b|
// (b = (D+m)^+ chi, A = (D+m)^+(D+m)) of psi = (psi_e, psi_o(psi_e)) -- see
// WEOOp::conv_site -- and that residual, in FP64, stops the solve and is
// reported.  The iterated Schur residual only triggers the checks: first at
// the Schur system's own tolerance, then at the level that the ratio of the
// two residuals seen at the last check predicts.
#include <cmath>
#include <vector>

#include "driver.cuh"

namespace swc {

template <typename T> __device__ __forceinline__ Sp<T> zero_sp() {
  Sp<T> a;
#pragma unroll
  for (int s = 0; s < 4; ++s) a.s[s] = zero3<T>();
  return a;
}

// Full index and coordinates of half-lattice site h of parity `par`.
__device__ __forceinline__ int half_site(const Geom& g, int h, int par, int x[4]) {
  coords(g, 2 * h, x);
  const int b = ((x[1] + x[2] + x[3]) & 1) ^ par;  // x0 of site 2h is even
  x[0] += b;
  return 2 * h + b;
}

// acc + sum_mu [(r - c g_mu) U_mu(x) psi(x+mu) + (r + c g_mu) U_mu(x-mu)^+ psi(x-mu)]
// at full site n; psi is read at the neighbours' half index (HALF) or full
// index from `in`.  c = -1 for the adjoint.
template <typename T, bool R1, bool HALF, typename G, typename In>
__device__ __forceinline__ Sp<T> wilson_hops(const Geom& g, int n, const int x[4], const G& U, const In& in, T r,
                                            bool dagger, Sp<T> acc) {
  const T sg = dagger ? T(-1) : T(1);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = hop(g, n, x, mu, +1), nb = hop(g, n, x, mu, -1);
    const bool ff = (mu == 3) && bc_flip(g, x, +1), fb = (mu == 3) && bc_flip(g, x, -1);
    {
      const M3<T> Uf = U.link(n, mu);
      const Sp<T> p = ld_sp<In, T>(in, HALF ? (nf >> 1) : nf);
      if (R1) {
        V3<T> h0, h1;
        wproject(mu, sg, p, h0, h1);
        V3<T> u0 = mv(Uf, h0), u1 = mv(Uf, h1);
        if (ff) { neg3(u0); neg3(u1); }
        wreconstruct(mu, sg, u0, u1, acc);
      } else {
        Sp<T> f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          f.s[k] = mv(Uf, p.s[k]);
          if (ff) neg3(f.s[k]);
        }
        wgeneral(mu, sg, r, f, acc);
      }
    }
    {
      const M3<T> Ub = U.link(nb, mu);
      const Sp<T> p = ld_sp<In, T>(in, HALF ? (nb >> 1) : nb);
      if (R1) {
        V3<T> h0, h1;
        wproject(mu, -sg, p, h0, h1);
        V3<T> u0 = mdv(Ub, h0), u1 = mdv(Ub, h1);
        if (fb) { neg3(u0); neg3(u1); }
        wreconstruct(mu, -sg, u0, u1, acc);
      } else {
        Sp<T> f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          f.s[k] = mdv(Ub, p.s[k]);
          if (fb) neg3(f.s[k]);
        }
        wgeneral(mu, -sg, r, f, acc);
      }
    }
  }
  return acc;
}

template <typename Op>
__global__ void __launch_bounds__(kTile) eo_prepass(Op op, typename Op::Vec in, size_t stride, const SysState* S,
                                                  int status, int dagger);

// The Schur operator D^ = M - D_eo D_oe / M on half-lattice fields, as an
// engine operator: apply() evaluates the even-site pass, prepass() launches
// the odd-site pass that fills the scratch it reads.
template <typename T, typename G, template <int> class VA, bool R1>
struct WEOOp {
  static constexpr int NC = 12;
  static constexpr int kMats = 4;
  static constexpr const char* kName = "wilson_eo";
  // per even site and application: both passes read every link of the lattice once
  static constexpr int kGaugeBytes = 4 * G::kBytes;
  static constexpr const char* kPrec = G::kPrec;
  static constexpr double kFlops = 2 * 1392.0;  // two half-lattice hopping terms per even site (Eq. 4)
  static constexpr bool kHalf = false;
  static constexpr bool kTwoPass = true;
  static constexpr int kNS = 1;
  // FP32 stencil blocks per SM: 7 (72 registers) with the spin-projected
  // hops, as the unpreconditioned operator; the full 4-spinor hops (r != 1)
  // need 96 registers not to spill
  static constexpr int kMinBlocks = R1 ? 7 : 5;
  using Vec = VA<12>;
  Geom full;         // the lattice
  G U;               // links of the full lattice
  size_t half_units;  // storage units of one half-lattice field (the offset of a system's scratch)
  double r;           // Wilson parameter (the pre-pass's hops)

  // Convergence on the full system: with psi_o rebuilt from psi_e the full
  // defect chi - (D+m) psi is (t, 0) with t = chi^_e - D^ psi_e, the Schur
  // defect, so the full normal-equation residual is
  //   |(D+m)^+ (t, 0)|^2 = M^2 |t|^2 (even sites) + |(D^+)_oe t|^2 (odd sites),
  // and (D^+)_oe t is what the adjoint pre-pass has left in t's scratch.
  static constexpr bool kFullConv = true;
  __device__ __forceinline__ double conv_site(int h, const Vec& t, double m, double r) const {
    const double M = 4.0 * r + m;
    const Sp<T> a = ld_sp<Vec, T>(t, h), u = ld_sp<Vec, T>(scratch(t), h);
    double e = 0.0, o = 0.0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        e += norm2(a.s[s].c[i]);
        o += norm2(u.s[s].c[i]);
      }
    return M * M * e + o;
  }

  __device__ __forceinline__ Vec scratch(const Vec& in) const {
    Vec u = in;
    u.p += half_units;
    return u;
  }
  // M in - D_eo u / M at even half-site h, u = D_oe in (or with the adjoint hops)
  __device__ __forceinline__ CV<T, 12> apply(const Geom&, int h, const Vec& in, T m, T r, bool dag) const {
    int x[4];
    const int n = half_site(full, h, 0, x);
    // M in + c hops(u) = c (2 M^2 in + hops(u)), c = 1 / (2M), with D_eo u =
    // -1/2 hops(u): one spinor accumulator, started from the site's own term
    const T M = T(4) * r + m, c = T(0.5) / M, M2 = T(2) * M * M;
    Sp<T> acc = ld_sp<Vec, T>(in, h);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) acc.s[s].c[i] = M2 * acc.s[s].c[i];
    acc = wilson_hops<T, R1, true>(full, n, x, U, scratch(in), r, dag, acc);
    CV<T, 12> v;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) v.c[3 * s + i] = c * acc.s[s].c[i];
    return v;
  }
  template <int NS, typename GG>
  __device__ __forceinline__ void apply_multi(const GG& g, int h, const Vec& in, size_t stride, unsigned act,
                                              const T* m, T r, bool dag, CV<T, 12>* out) const {
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (act & (1u << s)) out[s] = apply(full, h, sys_at(in, s, stride), m[s], r, dag);
  }
  // u = D_oe in (dagger: the adjoint hops) on the odd sites of the systems in
  // `status`, into each system's scratch
  void prepass(const Vec& in, size_t stride, const SysState* S, int status, int dagger, int cap,
               cudaStream_t st) const {
    const int gx = grid_for((const void*)eo_prepass<WEOOp>, kTile, full.V / 2, cap, (full.V / 2 + kTile - 1) / kTile);
    eo_prepass<WEOOp><<<dim3(gx, cap), kTile, 0, st>>>(*this, in, stride, S, status, dagger);
  }
  __device__ __forceinline__ void prepass_site(const Vec& in, int h, T r, bool dag) const {
    int x[4];
    const int n = half_site(full, h, 1, x);
    const Sp<T> hops = wilson_hops<T, R1, true>(full, n, x, U, in, r, dag, zero_sp<T>());
    CV<T, 12> v;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) v.c[3 * s + i] = T(-0.5) * hops.s[s].c[i];
    st_site(scratch(in), h, v);
  }
};

template <typename Op>
__global__ void __launch_bounds__(kTile) eo_prepass(Op op, typename Op::Vec in, size_t stride, const SysState* S,
                                                  int status, int dagger) {
  const int sys = blockIdx.y;
  if (S[sys].status != status) return;
  in = sys_view(in, sys, stride);
  using T = typename std::conditional<std::is_same<typename Op::Vec, VecC64<12>>::value, double, float>::type;
  const int Vh = op.full.V / 2;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x)
    op.prepass_site(in, h, (T)op.r, dagger != 0);
}

// chi^_e = chi_e - D_eo chi_o / M and the even part of the guess, per system,
// into half-lattice fields of stride s64 (FP64, canonical).
template <bool R1>
__global__ void eo_prepare(Geom g, const double2* U, const double2* chi, const double2* x, double2* chi_e,
                           double2* x_e, const double* mass, double r, size_t s64) {
  const int sys = blockIdx.y;
  const size_t full = (size_t)g.V * 12;
  chi += sys * full;
  x += sys * full;
  chi_e += sys * s64;
  x_e += sys * s64;
  const double M = 4.0 * r + mass[sys], c = 0.5 / M;
  const GaugeC64 Ug{U};
  const VecC64<12> in{const_cast<double2*>(chi)};
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.V / 2; h += gridDim.x * blockDim.x) {
    int xc[4];
    const int n = half_site(g, h, 0, xc);
    const Sp<double> hops = wilson_hops<double, R1, false>(g, n, xc, Ug, in, r, false, zero_sp<double>());
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int k = 3 * s + i;
        const double2 v = chi[(size_t)n * 12 + k];
        chi_e[(size_t)h * 12 + k] = make_double2(v.x + c * hops.s[s].c[i].re, v.y + c * hops.s[s].c[i].im);
        x_e[(size_t)h * 12 + k] = x[(size_t)n * 12 + k];
      }
  }
}

// psi_e into the even sites of x, psi_o = (chi_o - D_oe psi_e) / M into the odd ones.
template <bool R1>
__global__ void eo_rebuild(Geom g, const double2* U, const double2* chi, const double2* x_e, double2* x,
                           const double* mass, double r, size_t s64) {
  const int sys = blockIdx.y;
  const size_t full = (size_t)g.V * 12;
  chi += sys * full;
  x += sys * full;
  x_e += sys * s64;
  const double M = 4.0 * r + mass[sys], inv = 1.0 / M;
  const GaugeC64 Ug{U};
  const VecC64<12> in{const_cast<double2*>(x_e)};
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.V / 2; h += gridDim.x * blockDim.x) {
    int xc[4];
    const int ne = half_site(g, h, 0, xc);
#pragma unroll
    for (int k = 0; k < 12; ++k) x[(size_t)ne * 12 + k] = x_e[(size_t)h * 12 + k];
    const int no = half_site(g, h, 1, xc);
    const Sp<double> hops = wilson_hops<double, R1, true>(g, no, xc, Ug, in, r, false, zero_sp<double>());
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int k = 3 * s + i;
        const double2 v = chi[(size_t)no * 12 + k];  // D_oe psi_e = -1/2 hops
        x[(size_t)no * 12 + k] =
            make_double2((v.x + 0.5 * hops.s[s].c[i].re) * inv, (v.y + 0.5 * hops.s[s].c[i].im) * inv);
      }
  }
}

// Canonical FP64 vectors read as FP32 (the inner precision's view of chi).
template <int NC> struct VecC64as32 {
  double2* p;
  __device__ __forceinline__ cx<float> ld(int n, int c) const {
    const double2 v = __ldg(p + (size_t)n * NC + c);
    return {(float)v.x, (float)v.y};
  }
};

// |(D+m)^+ v|^2 per tile of kTile sites, one system per blockIdx.y, into
// part[sys * ntiles + tile] (a fixed summation order: tiles, then sum_tiles);
// v canonical FP64, the operator FP64 or the inner precision's
template <typename W>
__global__ void __launch_bounds__(kTile) eo_normal_norm(Geom g, W op, const double2* v, const double* mass,
                                                      double r, double* part, int ntiles) {
  __shared__ double sm[32];
  const int sys = blockIdx.y;
  const typename W::Vec in{const_cast<double2*>(v + sys * (size_t)g.V * 12)};
  const double m = mass[sys];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * kTile + threadIdx.x;
    double a = 0.0;
    if (n < g.V) {
      const auto w = op.apply(g, n, in, m, r, true);
#pragma unroll
      for (int c = 0; c < 12; ++c) a += norm2(w.c[c]);
    }
    a = block_sum(a, sm);
    if (threadIdx.x == 0) part[(size_t)sys * ntiles + tile] = a;
  }
}
static __global__ void __launch_bounds__(kTile) sum_tiles(const double* part, int ntiles, double* out) {
  __shared__ double sm[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < ntiles; i += blockDim.x) a += part[(size_t)blockIdx.x * ntiles + i];
  a = block_sum(a, sm);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

using WEO64R1 = WEOOp<double, GaugeC64, VecC64, true>;
using WEO64R = WEOOp<double, GaugeC64, VecC64, false>;
using WEO32R1 = WEOOp<float, GaugeP32, VecP32q, true>;
using WEO32R = WEOOp<float, GaugeP32, VecP32q, false>;

// |b|^2 = |(D+m)^+ chi|^2 of the full system for every system of the batch,
// into host h[nsys]: with the FP64 operator, or (u32: the packed FP32 links,
// lexicographic order) with the FP32 one -- the precision in which the
// mixed modes take every other system's |b|^2 (the tolerance's scale).
template <bool R1>
static int full_b2(const Geom& g, const SolveArgs& a, const double* dmass, const float2* u32,
                   std::vector<double>& h) {
  using W64 = WOp<double, GaugeC64, VecC64, R1>;
  using W32 = WOp<float, GaugeP32, VecC64as32, R1>;
  const int ntiles = (g.V + kTile - 1) / kTile;
  DevMem m;
  if (!m.alloc(sizeof(double) * ((size_t)ntiles + 1) * a.nsys, a.stream)) return SW_ERR_OOM;
  double* part = m.as<double>();
  double* nrm = part + (size_t)ntiles * a.nsys;
  const int gx = std::max(1, std::min(ntiles, sm_count() * 8 / std::max(1, a.nsys)));
  if (u32)
    eo_normal_norm<W32><<<dim3(gx, a.nsys), kTile, 0, a.stream>>>(g, W32{GaugeP32{u32}}, a.chi, dmass, a.r, part,
                                                                  ntiles);
  else
    eo_normal_norm<W64><<<dim3(gx, a.nsys), kTile, 0, a.stream>>>(g, W64{GaugeC64{a.U}}, a.chi, dmass, a.r, part,
                                                                  ntiles);
  sum_tiles<<<a.nsys, kTile, 0, a.stream>>>(part, ntiles, nrm);
  note_launches(2);
  h.assign(a.nsys, 0.0);
  if (const cudaError_t ce = cudaMemcpyAsync(h.data(), nrm, sizeof(double) * a.nsys, cudaMemcpyDeviceToHost,
                                             a.stream);
      ce != cudaSuccess)
    return cuda_fail(ce);
  if (const cudaError_t ce = cudaStreamSynchronize(a.stream); ce != cudaSuccess) return cuda_fail(ce);
  return SW_OK;
}

template <bool R1>
static int eo_solve(const Geom& g, const SolveArgs& a) {
  using D64 = WEOOp<double, GaugeC64, VecC64, R1>;
  using D32 = WEOOp<float, GaugeP32, VecP32q, R1>;
  const int Vh = g.V / 2;
  // one-dimensional layout geometry of the half lattice
  Geom gh{};
  gh.L[0] = Vh;
  gh.L[1] = gh.L[2] = gh.L[3] = 1;
  gh.stride[0] = 1;
  gh.stride[1] = gh.stride[2] = gh.stride[3] = Vh;
  gh.V = Vh;
  gh.apbc = 0;
  gh.shape = 0;
  const size_t nh = (size_t)Vh * 12, s64 = 2 * nh;
  DevMem fields, dmass;
  if (!fields.alloc(sizeof(double2) * s64 * 2 * a.nsys, a.stream) || !dmass.alloc(sizeof(double) * a.nsys, a.stream))
    return SW_ERR_OOM;
  double2* chi_e = fields.as<double2>();
  double2* x_e = chi_e + s64 * a.nsys;
  cudaMemcpyAsync(dmass.p, a.masses, sizeof(double) * a.nsys, cudaMemcpyHostToDevice, a.stream);
  const int gx = std::max(1, std::min((Vh + 127) / 128, sm_count() * 8 / std::max(1, a.nsys)));
  eo_prepare<R1><<<dim3(gx, a.nsys), 128, 0, a.stream>>>(g, a.U, a.chi, a.x, chi_e, x_e, dmass.as<double>(), a.r,
                                                         s64);
  note_launches(1);
  const D64 opd{g, GaugeC64{a.U}, nh, a.r};
  DevMem u32;
  D32 opf{};
  if (a.precision == SW_PREC_F32_RELIABLE) {
    if (!u32.alloc(sizeof(float2) * 36 * (size_t)g.V, a.stream)) return SW_ERR_OOM;
    pack_mats_p32<<<sm_count() * 8, 256, 0, a.stream>>>(make_blocked(g, 0), 4, a.U, u32.as<float2>());
    note_launches(1);
    opf = D32{g, GaugeP32{u32.as<float2>()}, VecP32q<12>::sys_units(Vh), a.r};
  }
  std::vector<double> b2;
  if (int e = full_b2<R1>(g, a, dmass.as<double>(), a.precision == SW_PREC_F32_RELIABLE ? u32.as<float2>() : nullptr,
                         b2))
    return e;
  SolveArgs ae = a;
  ae.chi = chi_e;
  ae.x = x_e;
  ae.conv_b2 = b2.data();
  const int rc = (a.precision == SW_PREC_F32_RELIABLE) ? run_cgne<D64, D32, true>(gh, opd, opf, ae)
                                                      : run_cgne<D64, D64, false>(gh, opd, opd, ae);
  if (rc < 0) return rc;
  eo_rebuild<R1><<<dim3(gx, a.nsys), 128, 0, a.stream>>>(g, a.U, a.chi, x_e, a.x, dmass.as<double>(), a.r, s64);
  note_launches(1);
  if (const cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e);
  return rc;
}

int wilson_cgne_eo(const Geom& g, const SolveArgs& a) {
  if (a.precision != SW_PREC_F64 && a.precision != SW_PREC_F32_RELIABLE) return SW_ERR_ARG;
  return (a.r == 1.0) ? eo_solve<true>(g, a) : eo_solve<false>(g, a);
}

}  // namespace swc
