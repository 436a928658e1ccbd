// FP64 fused multiply-add throughput of the current device (the denominator of
// the FP64 matvecs' roofline: the reliable updates' residuals are bound by the
// FP64 pipe, and the device's FP64 rate is not in its published bandwidth or
// tensor figures).  No counterpart in the paper.
#include <cuda_runtime.h>

#include "internal.h"

namespace swc {

constexpr int kChains = 8;  // independent FMA chains per thread (covers the pipe's latency)

// Each thread runs kChains dependent FMA chains of `iters` steps; the sum is
// stored so that no chain is dead code.
static __global__ void __launch_bounds__(256) dfma_chains(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace swc

using namespace swc;

extern "C" int sw_measure_fp64_peak(double* tflops, void* stream) {
  if (!tflops) return SW_ERR_NULL;
  *tflops = 0.0;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int per_sm = 0;
  if (const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_chains, 256, 0);
      e != cudaSuccess)
    return cuda_fail(e);
  const int blocks = sm_count() * (per_sm > 0 ? per_sm : 1), threads = 256, iters = 1 << 14;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(double) * blocks * threads, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_ms = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, st);
    dfma_chains<<<blocks, threads, 0, st>>>(out, iters, 1.0 - 1e-12, 1e-9);
    cudaEventRecord(e1, st);
    note_launches(1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (out) cudaFreeAsync(out, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e);
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = best_ms > 0.0 ? flops / (best_ms * 1e-3) / 1e12 : 0.0;
  return SW_OK;
}
