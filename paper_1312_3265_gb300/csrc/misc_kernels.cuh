// Layout conversion and small vector kernels used around the CG loop.
#pragma once
#include "cg_kernels.cuh"

namespace swc {

// canonical FP64 [V][nobj][9] -> planar FP32 [nobj*9][V]
static __global__ void pack_mats_p32(int V, int nobj, const double2* __restrict__ src, float2* __restrict__ dst) {
  const size_t total = (size_t)V * nobj * 9;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / ((size_t)nobj * 9);
    const size_t c = i - n * nobj * 9;
    const double2 v = src[i];
    dst[c * V + n] = make_float2((float)v.x, (float)v.y);
  }
}

// x64 (canonical) += x32 (planar); x32 = 0   -- systems with status NEED_RU
template <int NC>
__global__ void accum_x(int V, double2* x64, float2* x32, size_t s64, size_t s32, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_NEED_RU) return;
  x64 += sys * s64;
  x32 += sys * s32;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float2 a = x32[(size_t)c * V + n];
      double2 b = x64[(size_t)n * NC + c];
      b.x += (double)a.x;
      b.y += (double)a.y;
      x64[(size_t)n * NC + c] = b;
      x32[(size_t)c * V + n] = make_float2(0.f, 0.f);
    }
  }
}

// r32 (planar) = (float) r64 (canonical)   -- systems with status JUST_UPDATED
template <int NC>
__global__ void demote_r(int V, const double2* r64, float2* r32, size_t s64, size_t s32, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_JUST_UPDATED) return;
  r64 += sys * s64;
  r32 += sys * s32;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double2 a = r64[(size_t)n * NC + c];
      r32[(size_t)c * V + n] = make_float2((float)a.x, (float)a.y);
    }
  }
}

// Admission, step 1 (systems in ST_ADMIT): clear the search direction (and the
// FP32 correction), which may hold a previous system's values.
template <int NC, typename TP>
__global__ void admit_clear(int V, TP* p, float2* x32, size_t s, const SysState* S) {
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  p += sys * s;
  if (x32) x32 += sys * s;
  const size_t n = (size_t)V * NC;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    p[i] = TP{};
    if (x32) x32[i] = make_float2(0.f, 0.f);
  }
}

// Admission, step 3: |b|^2 and |x0|^2 of each admitted system -> S.b2, S.x02,
// S.tol2 <- S.tol2 * |b|^2 (S.tol2 holds tol^2 on entry), and the system's
// next state: b = 0 -> ST_ZERO_B, x0 = 0 -> ST_ZERO_GUESS, else ST_NEED_RU
// (non-finite b -> ST_FAILED).
template <int NC>
__global__ void __launch_bounds__(kTile) norm_b(int V, const double2* b, const double2* x, size_t s64, SysState* S,
                                               RedBuf rb) {
  __shared__ double sm[2 * 32];
  __shared__ int last;
  const int sys = blockIdx.y;
  if (S[sys].status != ST_ADMIT) return;
  b += sys * s64;
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
        const double2 v = b[(size_t)n * NC + c];
        const double2 w = x[(size_t)n * NC + c];
        acc[0] += v.x * v.x + v.y * v.y;
        acc[1] += w.x * w.x + w.y * w.y;
      }
    }
    block_sum_multi<2>(acc, sm);
    put_tile(rb, sys, tile, acc[0]);
    put_tile(rx, sys, tile, acc[1]);
  }
  if (block_done(rb, sys, &last)) {
    const double s = finalize_sum(rb, sys, ntiles, sm);
    const double sx = finalize_sum(rx, sys, ntiles, sm);
    if (threadIdx.x == 0) {
      SysState& st = S[sys];
      st.b2 = s;
      st.x02 = sx;
      st.tol2 *= s;
      if (!isfinite(s) || !isfinite(sx)) st.status = ST_FAILED;
      else if (s == 0.0) st.status = ST_ZERO_B;
      else if (sx == 0.0) st.status = ST_ZERO_GUESS;
      else st.status = ST_NEED_RU;
    }
  }
}

// Admission, step 4: b = 0 -> x = 0;  x0 = 0 -> r = b (exact initial residual).
template <int NC>
__global__ void admit_vectors(int V, double2* x, double2* r64, const double2* b64, size_t s64, const SysState* S) {
  const int sys = blockIdx.y;
  const int st = S[sys].status;
  if (st != ST_ZERO_B && st != ST_ZERO_GUESS) return;
  const size_t n = (size_t)V * NC, off = sys * s64;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (st == ST_ZERO_B) x[off + i] = make_double2(0.0, 0.0);
    else r64[off + i] = b64[off + i];
  }
}

// Admission, step 5: ST_ZERO_B -> converged; ST_ZERO_GUESS -> residual known.
static __global__ void admit_states(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  SysState& s = S[i];
  if (s.status == ST_ZERO_B) {
    s.rr_true = 0.0;
    s.status = ST_CONVERGED;
  } else if (s.status == ST_ZERO_GUESS) {
    s.rr = s.rr_true = s.rmax2 = s.b2;
    s.beta = 0.0;
    s.status = ST_JUST_UPDATED;
  }
}

// JUST_UPDATED -> RUNNING after the post-update p refresh
static __global__ void commit_status(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys && S[i].status == ST_JUST_UPDATED) S[i].status = ST_RUNNING;
}

}  // namespace swc
