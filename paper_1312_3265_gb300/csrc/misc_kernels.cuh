// Layout conversion and small vector kernels used around the CG loop.
#pragma once
#include "cg_kernels.cuh"

namespace swc {

// canonical FP64 [V][nobj][9] -> packed FP32 (nobj*9 planes), blocked site order
static __global__ void pack_mats_p32(GeomBlk gb, int nobj, const double2* __restrict__ src,
                                     float2* __restrict__ dst) {
  const int V = gb.V;
  const size_t total = (size_t)V * nobj * 9;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / ((size_t)nobj * 9);
    const size_t c = i - n * nobj * 9;
    const double2 v = src[i];
    dst[pk(lex_to_blk(gb, (int)n), nobj * 9, (int)c)] = make_float2((float)v.x, (float)v.y);
  }
}

// canonical FP64 links [V][4][9] -> packed FP16 12-real links (24 planes: rows 0, 1), blocked order
static __global__ void pack_links_h12(GeomBlk gb, const double2* __restrict__ src, __half2* __restrict__ dst) {
  const int V = gb.V;
  const size_t total = (size_t)V * 4 * 6;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / 24, r = i - n * 24, mu = r / 6, c = r - mu * 6;
    const double2 v = src[(n * 4 + mu) * 9 + c];
    dst[pk(lex_to_blk(gb, (int)n), 24, (int)(mu * 6 + c))] = __floats2half2_rn((float)v.x, (float)v.y);
  }
}

// canonical FP64 [V][nobj][9] -> packed FP16 (nobj*9 planes), blocked order
static __global__ void pack_mats_h(GeomBlk gb, int nobj, const double2* __restrict__ src,
                                   __half2* __restrict__ dst) {
  const int V = gb.V;
  const size_t total = (size_t)V * nobj * 9;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / ((size_t)nobj * 9);
    const size_t c = i - n * nobj * 9;
    const double2 v = src[i];
    dst[pk(lex_to_blk(gb, (int)n), nobj * 9, (int)c)] = __floats2half2_rn((float)v.x, (float)v.y);
  }
}

// Largest deviation of a link from SU(3): max over entries of |U U^+ - 1| and
// |det U - 1|, into *dev (as float bits; non-negative floats order like ints).
// The 12-real FP16 links rebuild the third row, which is exact only in SU(3).
static __global__ void su3_deviation(int V, const double2* __restrict__ U, unsigned* dev) {
  float worst = 0.f;
  for (size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x; l < (size_t)V * 4; l += (size_t)gridDim.x * blockDim.x) {
    const double2* q = U + l * 9;
    double a[3][3][2];
    for (int i = 0; i < 9; ++i) {
      a[i / 3][i % 3][0] = q[i].x;
      a[i / 3][i % 3][1] = q[i].y;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double re = 0, im = 0;
        for (int k = 0; k < 3; ++k) {  // (U U^+)_ij = sum_k U_ik conj(U_jk)
          re += a[i][k][0] * a[j][k][0] + a[i][k][1] * a[j][k][1];
          im += a[i][k][1] * a[j][k][0] - a[i][k][0] * a[j][k][1];
        }
        worst = fmaxf(worst, (float)hypot(re - (i == j), im));
      }
    // det = sum over the first row of U_0j times the cofactor
    double dre = 0, dim = 0;
    for (int j = 0; j < 3; ++j) {
      const int b = (j + 1) % 3, c = (j + 2) % 3;
      const double cre = a[1][b][0] * a[2][c][0] - a[1][b][1] * a[2][c][1] - (a[1][c][0] * a[2][b][0] - a[1][c][1] * a[2][b][1]);
      const double cim = a[1][b][0] * a[2][c][1] + a[1][b][1] * a[2][c][0] - (a[1][c][0] * a[2][b][1] + a[1][c][1] * a[2][b][0]);
      dre += a[0][j][0] * cre - a[0][j][1] * cim;
      dim += a[0][j][0] * cim + a[0][j][1] * cre;
    }
    worst = fmaxf(worst, (float)hypot(dre - 1.0, dim));
  }
  if (!(worst == worst)) worst = 3.0e38f;
  atomicMax(dev, __float_as_uint(worst));
}

// x64 (canonical) += x32 (packed, blocked order); x32 = 0   -- systems with status RU_PENDING
// (x32: the FP32 correction in its storage RV; s32 in RV's units)
template <int NC, typename RV>
__global__ void accum_x(GeomBlk gb, double2* x64, RV x32, size_t s64, size_t s32, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_RU_PENDING) return;
  const int V = gb.V;
  x64 += sys * s64;
  x32 = sys_view(x32, sys, s32);
  // component by component: each FP64 read-modify-write follows its own FP32
  // read (measured twice as fast as a whole-site FP32 read first)
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
    const int nb = lex_to_blk(gb, n);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const cx<float> a = x32.ld(nb, c);
      double2 b = x64[(size_t)n * NC + c];
      b.x += (double)a.re;
      b.y += (double)a.im;
      x64[(size_t)n * NC + c] = b;
      x32.st(nb, c, cx<float>{0.f, 0.f});
    }
  }
}

// r32 (packed, blocked order, storage RV) = (float) r64 (canonical)   -- systems with status JUST_UPDATED
template <int NC, typename RV>
__global__ void demote_r(GeomBlk gb, const double2* r64, RV r32, size_t s64, size_t s32, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_JUST_UPDATED) return;
  const int V = gb.V;
  r64 += sys * s64;
  r32 = sys_view(r32, sys, s32);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
    CV<float, NC> v;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double2 a = r64[(size_t)n * NC + c];
      v.c[c] = {(float)a.x, (float)a.y};
    }
    st_site(r32, lex_to_blk(gb, n), v);
  }
}

// Admission, step 1 (systems in ST_ADMIT): clear the search direction (and the
// FP32 correction), which may hold a previous system's values: every site of
// p through its accessor (paired layouts hold two systems in one unit), and
// xunits float2 of the correction.
template <typename PVec, int NC>
__global__ void admit_clear(int V, PVec p, size_t pstride, float2* x32, size_t xunits, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  p = sys_view(p, sys, pstride);
  if (x32) x32 += sys * xunits;
  using T = typename std::conditional<std::is_same<typename PVec::unit, double2>::value, double, float>::type;
  CV<T, NC> zero;
#pragma unroll
  for (int c = 0; c < NC; ++c) zero.c[c] = {T(0), T(0)};
  const size_t n = (size_t)V > xunits ? (size_t)V : xunits;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (i < (size_t)V) st_site(p, (int)i, zero);
    if (x32 && i < xunits) x32[i] = make_float2(0.f, 0.f);
  }
}

// Admission (mixed modes), before rhs_lo: chi (canonical FP64) -> its
// inner-precision copy in the stencil storage (blocked site order), for the
// systems in ST_ADMIT.
template <int NC, typename PVec>
__global__ void demote_chi(GeomBlk gb, const double2* chi, PVec out, size_t s64, size_t sout, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  chi += sys * s64;
  out = sys_view(out, sys, sout);
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gb.V; n += gridDim.x * blockDim.x) {
    CV<float, NC> v;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double2 a = chi[(size_t)n * NC + c];
      v.c[c] = {(float)a.x, (float)a.y};
    }
    st_site(out, lex_to_blk(gb, n), v);
  }
}

// Admission, step 3: |x0|^2 of each admitted system -> S.x02, and |b|^2 ->
// S.b2 from b (FP64 mode; b == nullptr: S.b2 already holds it, from rhs_lo);
// S.tol2 <- S.tol2 * |b|^2 (S.tol2 holds tol^2 on entry; |b|^2: S.cb2 when
// the criterion is another system's), S.trig2 <- tol^2 |b|^2, and the system's
// next state: b = 0 -> ST_ZERO_B, x0 = 0 -> ST_ZERO_GUESS, else ST_NEED_RU
// (non-finite b -> ST_FAILED).
template <int NC>
__global__ void __launch_bounds__(kTile) norm_b(int V, const double2* b, const double2* x, size_t s64, SysState* S,
                                               RedBuf rb) {
  __shared__ double sm[2 * 32];
  __shared__ int last;
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  if (b) b += sys * s64;
  x += sys * s64;
  const int ntiles = (V + kTile - 1) / kTile;
  RedBuf rx = rb;  // |x0|^2 tile sums go to the second half of the partials
  rx.partials += (size_t)gridDim.y * rb.pstride;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * kTile + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (n < V) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double2 w = x[(size_t)n * NC + c];
        acc[1] += w.x * w.x + w.y * w.y;
        if (b) {
          const double2 v = b[(size_t)n * NC + c];
          acc[0] += v.x * v.x + v.y * v.y;
        }
      }
    }
    block_sum_multi<2>(acc, sm);
    put_tile(rb, sys, tile, acc[0]);
    put_tile(rx, sys, tile, acc[1]);
  }
  if (block_done(rb, sys, &last, gridDim.x)) {
    const double s = b ? finalize_sum(rb, sys, ntiles, sm) : 0.0;
    const double sx = finalize_sum(rx, sys, ntiles, sm);
    if (threadIdx.x == 0) {
      SysState& st = S[sys];
      if (b) st.b2 = s;
      const double b2 = st.b2;
      st.x02 = sx;
      st.trig2 = st.tol2 * b2;
      st.tol2 *= st.cb2 > 0.0 ? st.cb2 : b2;
      if (!isfinite(b2) || !isfinite(sx)) st.status = ST_FAILED;
      else if (b2 == 0.0) st.status = ST_ZERO_B;
      else if (sx == 0.0) st.status = ST_ZERO_GUESS;
      else st.status = ST_NEED_RU;
    }
  }
}

// Admission, step 4: b = 0 -> x = 0;  x0 = 0 -> r = b (exact initial
// residual; FP64 mode: r64 = b64, mixed modes: rhs_lo has already stored r
// and p, b64 == nullptr).
template <int NC>
__global__ void admit_vectors(int V, double2* x, double2* r64, const double2* b64, size_t s64, const SysState* S) {
  const int sys = blockIdx.y;
  const int st = S[sys].status;
  if (st != ST_ZERO_B && (st != ST_ZERO_GUESS || !b64)) return;
  const size_t n = (size_t)V * NC, off = sys * s64;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (st == ST_ZERO_B) x[off + i] = make_double2(0.0, 0.0);
    else r64[off + i] = b64[off + i];
  }
}

// Admission, step 5: ST_ZERO_B -> converged; ST_ZERO_GUESS -> residual known:
// FP64 mode: JUST_UPDATED (p = r still to set); mixed modes (p_set): rhs_lo
// has set r = p = b, so the system runs at once.
static __global__ void admit_states(int nsys, SysState* S, int p_set) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  SysState& s = S[i];
  if (s.status == ST_ZERO_B) {
    s.rr_true = 0.0;
    s.status = ST_CONVERGED;
  } else if (s.status == ST_ZERO_GUESS) {
    s.rr = s.rr_true = s.rmax2 = s.b2;
    s.beta = 0.0;
    s.status = p_set ? ST_RUNNING : ST_JUST_UPDATED;
  }
}

// Start of a reliable update: NEED_RU -> RU_PENDING (the update's set).
static __global__ void mark_ru(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys && S[i].status == ST_NEED_RU) S[i].status = ST_RU_PENDING;
}

// End of a reliable update, after the p refresh: JUST_UPDATED -> READY.
static __global__ void mark_ready(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys && S[i].status == ST_JUST_UPDATED) S[i].status = ST_READY;
}

// First launch of every CG iteration, on the iteration stream: READY ->
// RUNNING.  A reliable update running concurrently on another stream marks
// its systems READY only after all its writes (x, r, p) are complete, and the
// switch happens between iterations, so every kernel of an iteration sees the
// same set of running systems.
static __global__ void commit_ready(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys && S[i].status == ST_READY) S[i].status = ST_RUNNING;
}

// Every system's status word <- st (set-up of the inner-precision apply).
static __global__ void set_status(int nsys, SysState* S, int st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys) S[i].status = st;
}

// Inner-precision field (packed, blocked order; the accessor's own reading,
// FP16 scales applied) -> canonical FP64, every system of the batch.
template <int NC, typename Vec>
__global__ void promote_vec(GeomBlk gb, Vec in, size_t sin, double2* out, size_t s64) {
  const int sys = blockIdx.y;
  in = sys_view(in, sys, sin);
  out += sys * s64;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gb.V; n += gridDim.x * blockDim.x) {
    const int nb = lex_to_blk(gb, n);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const cx<float> v = in.ld(nb, c);
      out[(size_t)n * NC + c] = make_double2((double)v.re, (double)v.im);
    }
  }
}

// End of a round of the device-driven solve: keep the loop of the solve's
// CUDA graph going while any system is in flight and fewer than max_rounds
// rounds have run; on the round cap, flag a timeout.  One block.
// ctl[0]: rounds run, ctl[1]: timeout flag.
static __global__ void round_end(int nsys, const SysState* S, int* ctl, int max_rounds,
                                 cudaGraphConditionalHandle loop) {
  __shared__ int busy;
  if (threadIdx.x == 0) busy = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nsys; i += blockDim.x) {
    const int s = S[i].status;
    if (s == ST_RUNNING || s == ST_NEED_RU || s == ST_JUST_UPDATED || s == ST_ADMIT || s == ST_ZERO_B ||
        s == ST_ZERO_GUESS || s == ST_RU_PENDING || s == ST_READY)
      busy = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int r = ++ctl[0];
    const bool cap = busy && r >= max_rounds;
    if (cap) ctl[1] = 1;
    cudaGraphSetConditional(loop, (busy && !cap) ? 1u : 0u);
  }
}

// n 8-byte words from src to dst.  Moves the solver's status words between
// the device and mapped pinned host memory: the kernel's loads and stores
// cross the host link directly, so these small transfers never queue behind
// the caller's bulk copies on a copy engine.
static __global__ void copy_words(const unsigned long long* __restrict__ src, unsigned long long* __restrict__ dst,
                                  size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace swc
