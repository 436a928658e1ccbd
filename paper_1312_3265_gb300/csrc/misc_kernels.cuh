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

// |b|^2 per system -> S.b2, and S.tol2 <- S.tol2 * |b|^2 (S.tol2 holds tol^2 on entry)
template <int NC>
__global__ void __launch_bounds__(kTile) norm_b(int V, const double2* b, size_t s64, SysState* S, RedBuf rb) {
  __shared__ double sm[32];
  __shared__ int last;
  const int sys = blockIdx.y;
  b += sys * s64;
  const int ntiles = (V + kTile - 1) / kTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int n = tile * kTile + threadIdx.x;
    double acc = 0.0;
    if (n < V) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const double2 v = b[(size_t)n * NC + c];
        acc += v.x * v.x + v.y * v.y;
      }
    }
    put_tile(rb, sys, tile, block_sum(acc, sm));
  }
  if (block_done(rb, sys, &last)) {
    const double s = finalize_sum(rb, sys, ntiles, sm);
    if (threadIdx.x == 0) {
      S[sys].b2 = s;
      S[sys].tol2 *= s;
    }
  }
}

// JUST_UPDATED -> RUNNING after the post-update p refresh
static __global__ void commit_status(int nsys, SysState* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsys && S[i].status == ST_JUST_UPDATED) S[i].status = ST_RUNNING;
}

}  // namespace swc
