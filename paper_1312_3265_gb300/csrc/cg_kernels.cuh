// CG kernels for CGNE (Eq. 2), generic over operator and storage.
//
// One iteration of textbook CG on A = (D+m)^+(D+m) takes three launches:
//   k1  t = (D+m) p,  pAp = <p, A p> = |t|^2,  alpha = |r|^2 / pAp
//   k2  Ap = (D+m)^+ t (never stored), r -= alpha Ap,
//       |r|^2, beta = |r_new|^2 / |r_old|^2, status decisions
//   k3  x += alpha p, then p = r + beta p (one read of the old p serves both)
// A system that k2 stops (for a reliable update) skips k3: its last
// x += alpha p is applied at the start of the update (k3 in its x-only form).
// Every launch covers a batch of independent systems (blockIdx.y = system)
// that share the gauge field; blocks of a system whose status is not RUNNING
// return at once, so converged systems cost nothing.  Scalars live in device
// memory (SysState), so the host never waits inside an iteration.
//
// Reductions: sites are cut into fixed tiles of kTile consecutive sites.  A
// tile's sum (each thread one site, promoted to FP64, warp shuffle + block
// tree) is stored as one double per tile; the last block of the system
// (atomic ticket) adds the tile sums in tile order.  The summation order thus
// depends only on the lattice volume -- not on the grid size, nor on which
// other systems share the launch -- so a system gives bit-identical results
// alone and in any batch.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "dslash.cuh"

namespace swc {

enum SysStatus : int {
  ST_RUNNING = 0,
  ST_NEED_RU = 1,       // host must recompute the FP64 residual
  ST_CONVERGED = 2,
  ST_FAILED = 3,        // NaN / breakdown
  ST_MAXITER = 4,
  ST_JUST_UPDATED = 5,  // residual replaced, p update pending
  ST_IDLE = 6,          // slot without a system
  ST_ADMIT = 7,         // slot being set up: b = (D+m)^+ chi, norms
  ST_ZERO_B = 8,        // admitted with b = 0: solution x = 0
  ST_ZERO_GUESS = 9,    // admitted with x0 = 0: r = b, no matvec needed
  ST_RU_PENDING = 10,   // taken into this round's reliable update (from NEED_RU)
  ST_READY = 11         // residual replaced and p refreshed: runs from the next iteration
};

// Plain data of 8-byte words (moved between device and host as such).
struct SysState {
  double rr;       // |r|^2 of the iterated residual
  double rr_old;   // previous |r|^2
  double pAp;
  double alpha;
  double beta;
  double b2;       // |b|^2
  double tol2;     // tol^2 |b|^2 (|b|^2: cb2 when set)
  double trig2;    // iterated |r|^2 at or below which a reliable update checks convergence
  double cb2;      // |b|^2 of the convergence criterion when it is another system's (0: b2)
  double rmax2;    // max |r|^2 since the last reliable update
  double delta2;   // reliable-update trigger factor (0: only at convergence)
  double rr_true;  // last FP64 residual norm^2
  double x02;      // |x0|^2 of the initial guess
  double mass;     // bare mass of this system
  int iter;
  int max_iter;
  int status;
  int n_ru;
};
static_assert(sizeof(SysState) % 8 == 0, "SysState moves as 8-byte words");

constexpr int kTile = 128;  // sites per reduction tile == threads per stencil block

struct RedBuf {
  double* partials;   // [nsys][pstride] tile sums
  unsigned* tickets;  // [nsys], zero between launches
  int pstride;        // >= kWarps x number of tiles (the iteration kernels' warp sums)
  double* hist;       // [nsys][kHist][2]: (alpha_k, beta_k) of every iteration, for Ritz values
};

constexpr int kHist = 4096;  // CG coefficients kept per system (Lanczos tridiagonal size cap)

__device__ __forceinline__ void record(const RedBuf& rb, int sys, int k, int which, double v) {
  if (rb.hist && k >= 0 && k < kHist) rb.hist[((size_t)sys * kHist + k) * 2 + which] = v;
}

__device__ __forceinline__ void put_tile(const RedBuf& rb, int sys, int tile, double v) {
  if (threadIdx.x == 0) rb.partials[(size_t)sys * rb.pstride + tile] = v;
}

// Sum the tile sums of system `sys` in a fixed order; valid in thread 0.
__device__ __forceinline__ double finalize_sum(const RedBuf& rb, int sys, int ntiles, double* smem) {
  const double* p = rb.partials + (size_t)sys * rb.pstride;
  double v = 0.0;
  for (int i = threadIdx.x; i < ntiles; i += blockDim.x) v += __ldcg(p + i);
  return block_sum(v, smem);
}

// Returns true in every thread of the block that is the last of the
// `nblocks` blocks of system (or group) `sys` to finish.
__device__ __forceinline__ bool block_done(const RedBuf& rb, int sys, int* flag_smem, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(rb.tickets + sys, 1u);
    *flag_smem = (t == nblocks - 1);
    if (*flag_smem) rb.tickets[sys] = 0u;
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

// ---------------------------------------------------------------- operator policies
template <typename T, int N> struct CV { cx<T> c[N]; };

template <typename T, typename G, typename Wt, template <int> class VA>
struct SWOp {
  static constexpr int NC = 3;
  static constexpr int kMats = 12;  // 4 links + 8 stored hypercube transports per site
  static constexpr const char* kName = "sw";
  static constexpr int kGaugeBytes = G::kBytes + Wt::kBytes;  // stored links + transports per site
  static constexpr double kFlops = 1743.0;  // per site and application (Eq. 4)
  static constexpr const char* kPrec = G::kPrec;
  static constexpr bool kHalf = std::is_same<G, GaugeP16>::value;  // FP16 storage
  // default systems per thread in the CG kernels (FP32 shares each matrix load
  // over several systems; FP64 is ALU-bound and gains nothing from it)
  static constexpr int kNS = sizeof(T) == 4 ? 4 : 1;
  using Vec = VA<3>;
  G U;
  Wt W;
  __device__ __forceinline__ CV<T, 3> apply(const Geom& g, int n, const Vec& in, T m, T r, bool dag) const {
    const V3<T> o = sw_site<T>(g, n, U, W, in, m, r, dag);
    CV<T, 3> v;
#pragma unroll
    for (int i = 0; i < 3; ++i) v.c[i] = o.c[i];
    return v;
  }
  template <int NS, typename GG>
  __device__ __forceinline__ void apply_multi(const GG& g, int n, const Vec& in, size_t stride, unsigned act,
                                              const T* m, T r, bool dag, CV<T, 3>* out) const {
    V3<T> o[NS];
    if constexpr (std::is_same<T, float>::value && NS % 2 == 0)
      sw_site_multi_pair<NS>(g, n, U, W, in, stride, act, m, r, dag, o);  // two systems per float2
    else
      sw_site_multi<T, NS>(g, n, U, W, in, stride, act, m, r, dag, o);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) out[s].c[i] = o[s].c[i];
  }
};

// LEAN: the spin-projected FP32 stencil in its lean form (wilson_site_lean) at
// 8 blocks per SM (64 registers), for lattices whose FP32 links stay in L2;
// beyond that the default form at 7 blocks, whose longer-lived loads keep
// more memory requests in flight per thread, is faster.  Both compute the
// same operations in the same order: their results are bit-identical.
template <typename T, typename G, template <int> class VA, bool R1, bool LEAN = false>
struct WOp {
  static constexpr int NC = 12;
  static constexpr int kMats = 4;   // 4 links per site
  static constexpr const char* kName = "wilson";
  static constexpr int kGaugeBytes = G::kBytes;
  static constexpr const char* kPrec = G::kPrec;
  static constexpr double kFlops = 1392.0;  // per site and application (Eq. 4)
  static constexpr bool kHalf = std::is_same<G, GaugeP16>::value;  // FP16 storage
  static constexpr int kNS = 1;
  static constexpr bool kLean =
      LEAN && R1 && std::is_same<G, GaugeP32>::value && std::is_same<VA<12>, VecP32q<12>>::value;
  static constexpr int kMinBlocks = kLean ? 8 : 0;
  using Vec = VA<12>;

  G U;
  __device__ __forceinline__ CV<T, 12> apply(const Geom& g, int n, const Vec& in, T m, T r, bool dag) const {
    const Sp<T> o = wilson_site<T, R1>(g, n, U, in, m, r, dag);
    CV<T, 12> v;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int i = 0; i < 3; ++i) v.c[3 * s + i] = o.s[s].c[i];
    return v;
  }
  template <int NS, typename GG>
  __device__ __forceinline__ void apply_multi(const GG& g, int n, const Vec& in, size_t stride, unsigned act,
                                              const T* m, T r, bool dag, CV<T, 12>* out) const {
    Sp<T> o[NS];
    if constexpr (NS == 1 && kLean)
      wilson_site_lean(g, n, U, in, m[0], dag, o[0]);
    else
      wilson_site_multi<T, R1, NS>(g, n, U, in, stride, act, m, r, dag, o);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) out[s].c[3 * k + i] = o[s].s[k].c[i];
  }
};

// Store a whole site: plain accessors component by component; FP16 vectors
// with the site's scale (largest |re|, |im|) so the halves hold psi/scale.
template <typename Vec, typename T, int NC>
__device__ __forceinline__ void st_site(const Vec& v, int n, const CV<T, NC>& a) {
#pragma unroll
  for (int c = 0; c < NC; ++c) v.st(n, c, a.c[c]);
}
template <int NC>
__device__ __forceinline__ void st_site(const VecP16<NC>& v, int n, const CV<float, NC>& a) {
  float m = 0.f;
#pragma unroll
  for (int c = 0; c < NC; ++c) m = fmaxf(m, fmaxf(fabsf(a.c[c].re), fabsf(a.c[c].im)));
  // Sites below 1e-30 (far tails of point-source solutions reach FP32
  // denormals, whose reciprocal overflows) are stored as exact zeros.
  if (!(m > 1e-30f)) m = (m == m) ? 0.f : m;
  const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
  for (int c = 0; c < NC; ++c) v.p[pk(n, NC, c)] = __floats2half2_rn(a.c[c].re * inv, a.c[c].im * inv);
  reinterpret_cast<float*>(v.p + (size_t)NC * v.V)[n] = m;
}

template <int NC>
__device__ __forceinline__ void st_site(const VecP32q<NC>& v, int n, const CV<float, NC>& a) {
#pragma unroll
  for (int q = 0; q < NC / 2; ++q)
    v.p[pk(n, NC / 2, q)] = make_float4(a.c[2 * q].re, a.c[2 * q].im, a.c[2 * q + 1].re, a.c[2 * q + 1].im);
}

// Load a whole site: plain accessors component by component; the float4
// layouts with one 16-byte load per pair of components.
template <typename Vec> struct SiteLoad {
  template <typename T, int NC> static __device__ __forceinline__ CV<T, NC> ld(const Vec& v, int n) {
    CV<T, NC> a;
#pragma unroll
    for (int c = 0; c < NC; ++c) a.c[c] = v.ld(n, c);
    return a;
  }
};
template <int NC> struct SiteLoad<VecP32q<NC>> {
  template <typename T, int N> static __device__ __forceinline__ CV<float, NC> ld(const VecP32q<NC>& v, int n) {
    CV<float, NC> a;
    const float4* b = v.p + pk(n, NC / 2, 0);
#pragma unroll
    for (int q = 0; q < NC / 2; ++q) {
      const float4 w = __ldg(b + q * 16);
      a.c[2 * q] = {w.x, w.y};
      a.c[2 * q + 1] = {w.z, w.w};
    }
    return a;
  }
};
template <typename T, int NC, typename Vec> __device__ __forceinline__ CV<T, NC> ld_site(const Vec& v, int n) {
  return SiteLoad<Vec>::template ld<T, NC>(v, n);
}

// FP32 residual / solution storage that goes with a stencil storage: the
// Wilson float4 planes keep r and x in float4 planes too (the r update of k2
// and the streaming k3 then move whole sites in 16-byte units, half the
// memory instructions of float2 planes); every other storage pairs with plain
// float2 planes.
template <typename VF, int NC> struct RVecOf { using type = VecP32<NC>; };
template <> struct RVecOf<VecP32q<12>, 12> { using type = VecP32q<12>; };

// Per-system view of a batched vector: system `sys` starts `sys * sstride`
// complex numbers after the base pointer (layout inside a system unchanged).
template <typename Vec> __device__ __forceinline__ Vec sys_view(Vec v, int sys, size_t sstride) {
  v.p += sys * sstride;
  return v;
}
template <int NC> __device__ __forceinline__ VecP32x2<NC> sys_view(VecP32x2<NC> v, int sys, size_t sstride) {
  return sys_at(v, sys, sstride);
}

struct BatchParams {
  double r;
  size_t sstride;      // units between systems: inner-precision r and x
  size_t sstride64;    // same for FP64 canonical vectors
  size_t vstride;      // same for the stencil vectors p and t
};

// (D+m) or (D+m)^+ at site n for the systems of a group selected by `act`
// (register-blocked: every gauge load is shared by the group's systems), each
// result handed to f(s, v).
template <int NS, typename Op, typename GG, typename T, typename F>
__device__ __forceinline__ void site_results(const Op& op, const GG& g, int n, const typename Op::Vec& in,
                                             size_t stride, unsigned act, const T* m, T r, bool dag, F&& f) {
  CV<T, Op::NC> v[NS];
  op.template apply_multi<NS, GG>(g, n, in, stride, act, m, r, dag, v);
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (act & (1u << s)) f(s, v[s]);
}

// ---------------------------------------------------------------- plain apply (ABI)
// out = (D+m) in, or (D+m)^+ in with dagger; with has_sub, out = sub - (D+m) in
// (the FP64 residual chi - (D+m) x of a reliable update).
template <typename T, typename Op>
__global__ void __launch_bounds__(kTile) apply_kernel(Geom g, Op op, typename Op::Vec in, typename Op::Vec out,
                                                    double mass0, size_t sstride, double r, int dagger,
                                                    const SysState* S, int only_status, int* nact = nullptr,
                                                    typename Op::Vec sub = {}, int has_sub = 0) {
  // mass: mass0, or each system's own mass when the launch is filtered by status;
  // nact (instrumentation, may be null) counts the systems computed
  const int sys = blockIdx.y;
  if (S && S[sys].status != only_status) return;
  if (nact && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nact, 1);
  in = sys_view(in, sys, sstride);
  out = sys_view(out, sys, sstride);
  if (has_sub) sub = sys_view(sub, sys, sstride);
  const T m = (T)(S ? S[sys].mass : mass0);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < g.V; n += gridDim.x * blockDim.x) {
    const CV<T, Op::NC> v = op.apply(g, n, in, m, (T)r, dagger != 0);
#pragma unroll
    for (int c = 0; c < Op::NC; ++c) out.st(n, c, has_sub ? sub.ld(n, c) - v.c[c] : v.c[c]);
  }
}

// Block-wide sums of NS doubles per thread (results valid in thread 0).
template <int NS> __device__ __forceinline__ void block_sum_multi(double* v, double* smem /* NS*32 */) {
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) smem[s * 32 + w] = v[s];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      v[s] = (lane < nw) ? smem[s * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
    }
  }
}

// The iteration kernels reduce without a block barrier per tile: each warp
// sums its 32 sites (FP64 shuffle tree) and lane 0 stores the warp sum at
// slot kWarps*tile + warp of the system's partials; the last block adds all
// kWarps*ntiles slots in slot order.  The order depends only on the volume,
// so a system's sums are the same whatever the grid or the batch.
constexpr int kWarps = kTile / 32;
template <int NS>
__device__ __forceinline__ void put_warp_sums(const RedBuf& rb, int sys0, unsigned act, int slot, double* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
    if (lane == 0 && (act & (1u << s))) rb.partials[(size_t)(sys0 + s) * rb.pstride + slot] = v[s];
  }
}

// Systems of group blockIdx.y that are RUNNING, as a bit mask, and their masses.
template <typename T, int NS>
__device__ __forceinline__ unsigned running_mask(const SysState* S, int sys0, int nsys, T* m) {
  unsigned act = 0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int sys = sys0 + s;
    m[s] = T(0);
    if (sys < nsys) {
      m[s] = (T)S[sys].mass;
      if (S[sys].status == ST_RUNNING) act |= 1u << s;
    }
  }
  return act;
}

// ---------------------------------------------------------------- k1: t = D p, |t|^2
// blockIdx.y = group of NS consecutive systems; tickets are per group.
// nact (instrumentation, may be null): the systems this launch computes are
// added to *nact, once per group.
// Minimum resident blocks per SM requested from the compiler for the
// inner-precision stencil kernels (caps their registers): they are
// latency-bound, so more resident warps hide more of the L2 latency
// (FP32 storage: staggered Wilson 9 blocks = 56 registers, Wilson 7 = 72 --
// 8 = 64 for its lean form on lattices whose links stay in L2 -- chosen from
// the spill counts of ptxas and GB300 timings).  The FP16-storage
// stencils also convert and scale every value they load: at 7 blocks they
// spill about 0.5 KB per thread (Wilson) and take 5 blocks (96 registers,
// no spills), staggered Wilson 7.  FP64 kernels are ALU-bound: no cap.
template <class Op, class = void> struct op_min_blocks : std::integral_constant<int, 0> {};
template <class Op> struct op_min_blocks<Op, std::void_t<decltype(Op::kMinBlocks)>>
    : std::integral_constant<int, Op::kMinBlocks> {};
template <typename T, typename Op> constexpr int stencil_min_blocks() {
  if (sizeof(T) != 4) return 1;
  if (op_min_blocks<Op>::value > 0) return op_min_blocks<Op>::value;  // the operator's own occupancy target
  if (Op::kHalf) return Op::NC == 3 ? 7 : 5;
  return Op::NC == 3 ? 9 : 7;
}

template <typename T, typename Op, int NS, typename GG>
__global__ void __launch_bounds__(kTile, stencil_min_blocks<T, Op>()) cg_k1(GG g, Op op, typename Op::Vec p, typename Op::Vec t,
                                               BatchParams bp, int nsys, SysState* S, RedBuf rb, int* nact,
                                               int gfast) {
  __shared__ double sm[NS * 32];
  __shared__ int last;
  // gfast: blockIdx.x = group of NS systems (the groups working on the same
  // tiles are launched side by side), blockIdx.y strides over the tiles;
  // otherwise the other way round
  const int grp = gfast ? blockIdx.x : blockIdx.y, bt = gfast ? blockIdx.y : blockIdx.x;
  const int nbt = gfast ? gridDim.y : gridDim.x;
  const int sys0 = grp * NS;
  T m[NS];
  const unsigned act = running_mask<T, NS>(S, sys0, nsys, m);
  if (!act) return;
  if (nact && bt == 0 && threadIdx.x == 0) atomicAdd(nact, __popc(act));
  p = sys_view(p, sys0, bp.vstride);
  t = sys_view(t, sys0, bp.vstride);
  const int ntiles = (g.V + kTile - 1) / kTile;
  // grid-stride over tiles: the blocks resident at a time cover neighbouring
  // tiles, which keeps their neighbour reads together in L2 (measured faster
  // on GB300 than giving each block one contiguous range of tiles)
  for (int tile = bt; tile < ntiles; tile += nbt) {
    const int n = tile * kTile + threadIdx.x;
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    if (n < g.V) {
      site_results<NS>(op, g, n, p, bp.vstride, act, m, (T)bp.r, false, [&](int s, const CV<T, Op::NC>& v) {
        st_site(sys_at(t, s, bp.vstride), n, v);
        T a = T(0);
#pragma unroll
        for (int c = 0; c < Op::NC; ++c) a += norm2(v.c[c]);
        acc[s] = (double)a;
      });
    }
    put_warp_sums<NS>(rb, sys0, act, kWarps * tile + (threadIdx.x >> 5), acc);
  }
  __threadfence();  // every warp's partials, before the block's ticket
  if (block_done(rb, grp, &last, nbt)) {
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      if (!(act & (1u << s))) continue;
      const int sys = sys0 + s;
      const double pAp = finalize_sum(rb, sys, kWarps * ntiles, sm);
      if (threadIdx.x == 0) {
        SysState& st = S[sys];
        st.pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp)) {
          st.status = ST_FAILED;
        } else {
          st.alpha = st.rr / pAp;
          record(rb, sys, st.iter, 0, st.alpha);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- k2: Ap = D^+ t; x, r update; |r|^2
template <typename T, typename Op, int NS, typename RVec, typename GG>
__global__ void __launch_bounds__(kTile, stencil_min_blocks<T, Op>()) cg_k2(GG g, Op op, typename Op::Vec t, RVec r,
                                               BatchParams bp, int nsys, SysState* S, RedBuf rb,
                                               int* nact, int gfast) {
  __shared__ double sm[NS * 32];
  __shared__ int last;
  // groups and tiles as in cg_k1
  const int grp = gfast ? blockIdx.x : blockIdx.y, bt = gfast ? blockIdx.y : blockIdx.x;
  const int nbt = gfast ? gridDim.y : gridDim.x;
  const int sys0 = grp * NS;
  T m[NS];
  const unsigned act = running_mask<T, NS>(S, sys0, nsys, m);
  if (!act) return;
  if (nact && bt == 0 && threadIdx.x == 0) atomicAdd(nact, __popc(act));
  T alpha[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) alpha[s] = (act & (1u << s)) ? (T)S[sys0 + s].alpha : T(0);
  t = sys_view(t, sys0, bp.vstride);
  r = sys_view(r, sys0, bp.sstride);
  const int ntiles = (g.V + kTile - 1) / kTile;
  for (int tile = bt; tile < ntiles; tile += nbt) {
    const int n = tile * kTile + threadIdx.x;
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    if (n < g.V) {
      site_results<NS>(op, g, n, t, bp.vstride, act, m, (T)bp.r, true, [&](int s, const CV<T, Op::NC>& ap) {
        const RVec rs = sys_at(r, s, bp.sstride);
        CV<T, Op::NC> rv = ld_site<T, Op::NC>(rs, n);
        T a = T(0);
#pragma unroll
        for (int c = 0; c < Op::NC; ++c) {
          rv.c[c] = rv.c[c] - alpha[s] * ap.c[c];
          a += norm2(rv.c[c]);
        }
        st_site(rs, n, rv);
        acc[s] = (double)a;
      });
    }
    put_warp_sums<NS>(rb, sys0, act, kWarps * tile + (threadIdx.x >> 5), acc);
  }
  __threadfence();  // every warp's partials, before the block's ticket
  if (block_done(rb, grp, &last, nbt)) {
#pragma unroll 1
    for (int s = 0; s < NS; ++s) {
      if (!(act & (1u << s))) continue;
      const int sys = sys0 + s;
      const double rr = finalize_sum(rb, sys, kWarps * ntiles, sm);
      if (threadIdx.x == 0) {
        SysState& st = S[sys];
        st.iter += 1;
        if (!isfinite(rr)) {
          st.status = ST_FAILED;
        } else {
          st.rr_old = st.rr;
          st.rr = rr;
          st.beta = rr / st.rr_old;
          record(rb, sys, st.iter - 1, 1, st.beta);
          if (rr > st.rmax2) st.rmax2 = rr;
          if (rr <= st.trig2 || st.iter >= st.max_iter || rr < st.delta2 * st.rmax2) st.status = ST_NEED_RU;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- k3: x += alpha p, p = r + beta p
// mode bit 1: x += alpha p (the iteration's solution update, deferred from
// k2 so that one read of p serves it and the new direction); bit 2:
// p = r + beta p.  Systems in ST_RUNNING take both, a reliable update takes
// the x part first (systems in ST_RU_PENDING) and the p part last (ST_JUST_UPDATED).
template <typename T, typename RVec, typename PVec, int NC>
__global__ void __launch_bounds__(256) cg_k3(int V, RVec r, PVec p, RVec x, size_t rstride, size_t pstride,
                                             const SysState* S, int only_status, int mode, int* nact = nullptr) {
  const int sys = blockIdx.y;
  if (S[sys].status != only_status) return;
  if (nact && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nact, 1);
  r = sys_view(r, sys, rstride);
  p = sys_view(p, sys, pstride);
  x = sys_view(x, sys, rstride);
  const T beta = (T)S[sys].beta, alpha = (T)S[sys].alpha;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
    const CV<T, NC> po = ld_site<T, NC>(p, n);
    if (mode & 1) {
      CV<T, NC> xv = ld_site<T, NC>(x, n);
#pragma unroll
      for (int c = 0; c < NC; ++c) xv.c[c] = xv.c[c] + alpha * po.c[c];
      st_site(x, n, xv);
    }
    if (mode & 2) {
      CV<T, NC> v = ld_site<T, NC>(r, n);
#pragma unroll
      for (int c = 0; c < NC; ++c) v.c[c] = v.c[c] + beta * po.c[c];
      st_site(p, n, v);
    }
  }
}

// k3 for a paired p (two systems' lanes per 16-byte unit): one thread per
// site and pair reads the pair's unit once for both systems.  A lane whose
// system is in another state keeps its value: when only one lane is active,
// only its words are stored (another stream may be writing the other
// lane's); with both active the whole unit is.
template <typename RVec, typename PVec, int NC>
__global__ void __launch_bounds__(256) cg_k3_pair(int V, RVec r, PVec p, RVec x, size_t rstride, size_t pstride,
                                                  const SysState* S, int nsys, int only_status, int mode,
                                                  int* nact = nullptr) {
  const int s0 = 2 * blockIdx.y;
  const bool a0 = S[s0].status == only_status, a1 = s0 + 1 < nsys && S[s0 + 1].status == only_status;
  if (!a0 && !a1) return;
  if (nact && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nact, (int)a0 + (int)a1);
  float4* pp = p.p + (size_t)blockIdx.y * 2 * pstride;
  const RVec r0 = sys_view(r, s0, rstride), x0 = sys_view(x, s0, rstride);
  const RVec r1 = sys_view(r, a1 ? s0 + 1 : s0, rstride), x1 = sys_view(x, a1 ? s0 + 1 : s0, rstride);
  const float beta0 = (float)S[s0].beta, alpha0 = (float)S[s0].alpha;
  const float beta1 = a1 ? (float)S[s0 + 1].beta : 0.f, alpha1 = a1 ? (float)S[s0 + 1].alpha : 0.f;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float4* u = pp + pk(n, NC, c);
      const float4 w = *u;  // (s0.re, s1.re, s0.im, s1.im)
      if (mode & 1) {
        if (a0) {
          const cx<float> xv = x0.ld(n, c);
          x0.st(n, c, {xv.re + alpha0 * w.x, xv.im + alpha0 * w.z});
        }
        if (a1) {
          const cx<float> xv = x1.ld(n, c);
          x1.st(n, c, {xv.re + alpha1 * w.y, xv.im + alpha1 * w.w});
        }
      }
      if (mode & 2) {
        float4 o = w;
        if (a0) {
          const cx<float> rv = r0.ld(n, c);
          o.x = rv.re + beta0 * w.x;
          o.z = rv.im + beta0 * w.z;
        }
        if (a1) {
          const cx<float> rv = r1.ld(n, c);
          o.y = rv.re + beta1 * w.y;
          o.w = rv.im + beta1 * w.w;
        }
        if (a0 && a1) {
          *u = o;
        } else {
          float* q = reinterpret_cast<float*>(u) + (a0 ? 0 : 1);
          q[0] = a0 ? o.x : o.y;
          q[2] = a0 ? o.z : o.w;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- FP64 residual (reliable update)
// A reliable update acts on the systems in ST_RU_PENDING (marked from
// ST_NEED_RU by the host's round, so that iterations running at the same time
// on another stream -- which may move other systems to ST_NEED_RU -- cannot
// change the set while the update's kernels run).  It ends in ST_READY;
// commit_ready, launched on the iteration stream at an iteration boundary,
// lets the system run again.
// r64 = (D+m)^+ t64 with t64 = chi - (D+m) x (apply_kernel's has_sub form), so
// r64 = b - A x for b = (D+m)^+ chi; |r64|^2, then the convergence decision.
// An operator with a full-system criterion (full_conv) also sums its
// conv_site over the sites; that sum, not |r64|^2, decides convergence and is
// reported, and a system that reached its trigger without converging gets
// the trigger tightened by the ratio the two sums showed.
template <class Op, class = void> struct full_conv : std::false_type {};
template <class Op> struct full_conv<Op, std::void_t<decltype(Op::kFullConv)>> : std::bool_constant<Op::kFullConv> {};

template <typename Op>
__global__ void __launch_bounds__(kTile) residual64(Geom g, Op op, typename Op::Vec t, typename Op::Vec r,
                                                  BatchParams bp, SysState* S, RedBuf rb, int* nact = nullptr) {
  constexpr bool kConv = full_conv<Op>::value;
  __shared__ double sm[(kConv ? 2 : 1) * 32];
  __shared__ int last;
  const int sys = blockIdx.y;
  if (S[sys].status != ST_RU_PENDING) return;
  if (nact && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nact, 1);
  t = sys_view(t, sys, bp.sstride64);
  r = sys_view(r, sys, bp.sstride64);
  const double m = S[sys].mass;
  const int ntiles = (g.V + kTile - 1) / kTile;
  RedBuf rc = rb;  // the criterion's tile sums: the second half of the partials
  rc.partials += (size_t)gridDim.y * rb.pstride;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * kTile + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (n < g.V) {
      const CV<double, Op::NC> at = op.apply(g, n, t, m, bp.r, true);
#pragma unroll
      for (int c = 0; c < Op::NC; ++c) {
        r.st(n, c, at.c[c]);
        acc[0] += norm2(at.c[c]);
      }
      if constexpr (kConv) acc[1] = op.conv_site(n, t, m, bp.r);
    }
    if constexpr (kConv) {
      block_sum_multi<2>(acc, sm);
      put_tile(rb, sys, tile, acc[0]);
      put_tile(rc, sys, tile, acc[1]);
    } else {
      put_tile(rb, sys, tile, block_sum(acc[0], sm));
    }
  }
  if (block_done(rb, sys, &last, gridDim.x)) {
    const double rr = finalize_sum(rb, sys, ntiles, sm);
    double conv = rr;
    if constexpr (kConv) conv = finalize_sum(rc, sys, ntiles, sm);
    if (threadIdx.x == 0) {
      SysState& s = S[sys];
      s.rr_true = conv;
      s.n_ru += 1;
      if (!isfinite(rr) || !isfinite(conv)) {
        s.status = ST_FAILED;
      } else if (conv <= s.tol2) {
        s.status = ST_CONVERGED;
      } else if (s.iter >= s.max_iter) {
        s.status = ST_MAXITER;
      } else {
        // (conv > tol2 here, so the new trigger is below rr)
        if constexpr (kConv) s.trig2 = 0.8 * rr * (s.tol2 / conv);
        s.beta = (s.iter == 0) ? 0.0 : rr / s.rr_old;
        record(rb, sys, s.iter - 1, 1, s.beta);
        s.rr = rr;
        s.rmax2 = rr;
        s.status = ST_JUST_UPDATED;
      }
    }
  }
}

// ---------------------------------------------------------------- inner-precision right-hand side
// Admission in the mixed modes (systems in ST_ADMIT): b = (D+m)^+ chi with the
// inner-precision operator on chi's inner-precision copy (in the stencil
// storage), stored as the iterated residual r and as the first search
// direction p (x0 = 0 gives r0 = p0 = b), and |b|^2 (FP64 accumulation) ->
// S.b2.  b is needed only as the iteration's starting residual and for the
// tolerance scale: every residual that decides convergence is recomputed in
// FP64 from chi itself (residual64), so no FP64 copy of b exists.
template <typename T, typename Op, typename RVec, typename GG>
__global__ void __launch_bounds__(kTile) rhs_lo(GG g, Op op, typename Op::Vec chi, typename Op::Vec p, RVec r,
                                              BatchParams bp, SysState* S, RedBuf rb, int* nact = nullptr) {
  __shared__ double sm[32];
  __shared__ int last;
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  if (nact && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(nact, 1);
  chi = sys_view(chi, sys, bp.vstride);
  p = sys_view(p, sys, bp.vstride);
  r = sys_view(r, sys, bp.sstride);
  const T m = (T)S[sys].mass;
  const int ntiles = (g.V + kTile - 1) / kTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * kTile + threadIdx.x;
    double acc = 0.0;
    if (n < g.V) {
      CV<T, Op::NC> v;
      op.template apply_multi<1, GG>(g, n, chi, bp.vstride, 1u, &m, (T)bp.r, true, &v);
      T a = T(0);
#pragma unroll
      for (int c = 0; c < Op::NC; ++c) a += norm2(v.c[c]);
      st_site(r, n, v);
      st_site(p, n, v);
      acc = (double)a;
    }
    put_tile(rb, sys, tile, block_sum(acc, sm));
  }
  if (block_done(rb, sys, &last, gridDim.x)) {
    const double b2 = finalize_sum(rb, sys, ntiles, sm);
    if (threadIdx.x == 0) S[sys].b2 = b2;
  }
}

}  // namespace swc
