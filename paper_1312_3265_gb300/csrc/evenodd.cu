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
// carry the full lattice geometry for their neighbours.  Convergence: the
// engine stops on the FP64 normal-equation residual of the Schur system; the
// solution is then rebuilt on the full lattice and the FP64 normal-equation
// residual of the full system, |b - A psi| / |b| with b = (D+m)^+ chi, is
// recomputed and reported.  A system whose full residual is above the
// tolerance resumes the Schur solve from its solution with a proportionally
// tighter tolerance (at most four passes); the others stop at admission with
// their solution unchanged, so each system's result does not depend on the
// batch (its reliable-update count includes those admission residuals).
#include <cmath>
#include <vector>

#include "driver.cuh"

namespace swc {

// Full index and coordinates of half-lattice site h of parity `par`.
__device__ __forceinline__ int half_site(const Geom& g, int h, int par, int x[4]) {
  coords(g, 2 * h, x);
  const int b = ((x[1] + x[2] + x[3]) & 1) ^ par;  // x0 of site 2h is even
  x[0] += b;
  return 2 * h + b;
}

// sum_mu [(r - c g_mu) U_mu(x) psi(x+mu) + (r + c g_mu) U_mu(x-mu)^+ psi(x-mu)]
// at full site n; psi is read at the neighbours' half index (HALF) or full
// index from `in`.  c = -1 for the adjoint.
template <typename T, bool R1, bool HALF, typename G, typename In>
__device__ __forceinline__ Sp<T> wilson_hops(const Geom& g, int n, const int x[4], const G& U, const In& in, T r,
                                            bool dagger) {
  Sp<T> acc;
#pragma unroll
  for (int s = 0; s < 4; ++s) acc.s[s] = zero3<T>();
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
  using Vec = VA<12>;
  Geom full;         // the lattice
  G U;               // links of the full lattice
  size_t half_units;  // storage units of one half-lattice field (the offset of a system's scratch)
  double r;           // Wilson parameter (the pre-pass's hops)

  __device__ __forceinline__ Vec scratch(const Vec& in) const {
    Vec u = in;
    u.p += half_units;
    return u;
  }
  // M in - D_eo u / M at even half-site h, u = D_oe in (or with the adjoint hops)
  __device__ __forceinline__ CV<T, 12> apply(const Geom&, int h, const Vec& in, T m, T r, bool dag) const {
    int x[4];
    const int n = half_site(full, h, 0, x);
    const Sp<T> hops = wilson_hops<T, R1, true>(full, n, x, U, scratch(in), r, dag);
    const Sp<T> self = ld_sp<Vec, T>(in, h);
    const T M = T(4) * r + m, c = T(0.5) / M;  // D_eo u = -1/2 hops(u)
    CV<T, 12> v;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) v.c[3 * s + i] = M * self.s[s].c[i] + c * hops.s[s].c[i];
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
    const Sp<T> hops = wilson_hops<T, R1, true>(full, n, x, U, in, r, dag);
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
    const Sp<double> hops = wilson_hops<double, R1, false>(g, n, xc, Ug, in, r, false);
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
    const Sp<double> hops = wilson_hops<double, R1, true>(g, no, xc, Ug, in, r, false);
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

// |v|^2 per system in a fixed order: tile sums, then one block per system.
static __global__ void __launch_bounds__(kTile) tile_norms(const double2* v, size_t n, size_t stride, double* part,
                                                         int ntiles) {
  __shared__ double sm[32];
  const int sys = blockIdx.y;
  v += sys * stride;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    double a = 0.0;
    for (size_t i = (size_t)t * kTile * 12 + threadIdx.x; i < std::min(n, (size_t)(t + 1) * kTile * 12);
         i += blockDim.x)
      a += v[i].x * v[i].x + v[i].y * v[i].y;
    a = block_sum(a, sm);
    if (threadIdx.x == 0) part[(size_t)sys * ntiles + t] = a;
  }
}
static __global__ void __launch_bounds__(kTile) sum_tiles(const double* part, int ntiles, double* out) {
  __shared__ double sm[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < ntiles; i += blockDim.x) a += part[(size_t)blockIdx.x * ntiles + i];
  a = block_sum(a, sm);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}
// out = a - b
static __global__ void sub_fields(const double2* a, const double2* b, double2* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

using WEO64R1 = WEOOp<double, GaugeC64, VecC64, true>;
using WEO64R = WEOOp<double, GaugeC64, VecC64, false>;
using WEO32R1 = WEOOp<float, GaugeP32, VecP32q, true>;
using WEO32R = WEOOp<float, GaugeP32, VecP32q, false>;

// FP64 normal-equation residual |b - A psi| / |b| of the full system for every
// system of the batch (b = (D+m)^+ chi, A = (D+m)^+(D+m)).
static int full_residuals(const Geom& g, const SolveArgs& a, std::vector<double>& out) {
  const size_t n = (size_t)g.V * 12;
  const int ntiles = (g.V + kTile - 1) / kTile;
  DevMem m;
  if (!m.alloc(sizeof(double2) * n * 4 + sizeof(double) * (size_t)ntiles * 2 + 2 * sizeof(double), a.stream))
    return SW_ERR_OOM;
  double2 *t = m.as<double2>(), *u = t + n, *b = u + n, *rr = b + n;
  double* part = reinterpret_cast<double*>(rr + n);
  double* nrm = part + 2 * (size_t)ntiles;
  out.assign(a.nsys, 0.0);
  for (int i = 0; i < a.nsys; ++i) {
    const double2* chi = a.chi + (size_t)i * n;
    const double2* x = a.x + (size_t)i * n;
    int e;
    if ((e = wilson_apply_f64(g, a.U, x, t, a.masses[i], a.r, 0, a.stream))) return e;  // (D+m) psi
    sub_fields<<<sm_count() * 4, 256, 0, a.stream>>>(chi, t, u, n);                     // chi - (D+m) psi
    if ((e = wilson_apply_f64(g, a.U, u, rr, a.masses[i], a.r, 1, a.stream))) return e;  // b - A psi
    if ((e = wilson_apply_f64(g, a.U, chi, b, a.masses[i], a.r, 1, a.stream))) return e;  // b
    tile_norms<<<dim3(std::min(ntiles, sm_count() * 8), 1), kTile, 0, a.stream>>>(rr, n, 0, part, ntiles);
    tile_norms<<<dim3(std::min(ntiles, sm_count() * 8), 1), kTile, 0, a.stream>>>(b, n, 0, part + ntiles, ntiles);
    sum_tiles<<<2, kTile, 0, a.stream>>>(part, ntiles, nrm);
    note_launches(5);
    double h[2] = {0.0, 0.0};
    if (const cudaError_t ce = cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, a.stream);
        ce != cudaSuccess)
      return cuda_fail(ce);
    if (const cudaError_t ce = cudaStreamSynchronize(a.stream); ce != cudaSuccess) return cuda_fail(ce);
    out[i] = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  }
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
  SolveArgs ae = a;
  ae.chi = chi_e;
  ae.x = x_e;
  std::vector<sw_solve_info> infos(a.nsys), total(a.nsys);
  ae.infos = infos.data();
  std::vector<double> res, tols(a.nsys, a.tol);
  ae.tols = tols.data();
  int rc = SW_OK;
  for (int pass = 0; pass < 4; ++pass) {
    rc = (a.precision == SW_PREC_F32_RELIABLE) ? run_cgne<D64, D32, true>(gh, opd, opf, ae)
                                               : run_cgne<D64, D64, false>(gh, opd, opd, ae);
    if (rc < 0) return rc;
    for (int i = 0; i < a.nsys; ++i) {
      total[i].iters += infos[i].iters;
      total[i].reliable_updates += infos[i].reliable_updates;
      if (pass == 0 || total[i].lambda_max == 0.0) {  // the Ritz values of the main pass
        total[i].lambda_min = infos[i].lambda_min;
        total[i].lambda_max = infos[i].lambda_max;
      }
    }
    eo_rebuild<R1><<<dim3(gx, a.nsys), 128, 0, a.stream>>>(g, a.U, a.chi, x_e, a.x, dmass.as<double>(), a.r, s64);
    note_launches(1);
    if (int e = full_residuals(g, a, res)) return e;
    bool again = false;
    for (int i = 0; i < a.nsys; ++i)
      if (res[i] > a.tol) {  // this system resumes from its psi_e with a tighter Schur tolerance
        tols[i] = std::max(1e-15, tols[i] * 0.5 * a.tol / res[i]);
        again = true;
      }
    // (a system already within tol is re-admitted with its own tolerance and
    // stops at admission, x unchanged: its result does not depend on the batch)
    if (rc != SW_OK || !again) break;
  }
  int worst_rc = rc;
  for (int i = 0; i < a.nsys; ++i) {
    if (rc == SW_OK && !(res[i] <= a.tol)) worst_rc = worst_code(worst_rc, SW_NOT_CONVERGED);
    if (a.infos) {
      sw_solve_info& o = a.infos[i];
      o = total[i];
      o.status = rc != SW_OK ? infos[i].status : (res[i] <= a.tol ? SW_OK : SW_NOT_CONVERGED);
      o.precision = a.precision;
      o.true_rel_resid = res[i];
    }
  }
  return worst_rc;
}

int wilson_cgne_eo(const Geom& g, const SolveArgs& a) {
  if (a.precision != SW_PREC_F64 && a.precision != SW_PREC_F32_RELIABLE) return SW_ERR_ARG;
  return (a.r == 1.0) ? eo_solve<true>(g, a) : eo_solve<false>(g, a);
}

}  // namespace swc
