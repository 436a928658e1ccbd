// Internal C++ entry points behind the C ABI (one translation unit per operator).
#pragma once
#include <cuda_runtime.h>
#include "../../include/sw_cgne.h"

namespace swc {

struct Geom;

// Common arguments of a batched CGNE call.  chi, x: nsys systems back to back
// in the canonical layout.  masses: host array [nsys].  infos: host [nsys].
struct SolveArgs {
  const double2* U;
  const double2* W;  // staggered Wilson only
  const double2* chi;
  double2* x;
  int nsys;
  const double* masses;
  double r;
  double tol;
  int max_iter;
  int precision;
  sw_solve_info* infos;
  cudaStream_t stream;
  const double* tols = nullptr;  // host [nsys]: per-system tolerances (nullptr: tol for every system)
  const double* conv_b2 = nullptr;  // host [nsys]: |b|^2 of an operator's own convergence criterion
};

int hypercube_build_f64(const Geom& g, const double2* U, double2* W, cudaStream_t st);
int sw_apply_f64(const Geom& g, const double2* U, const double2* W, const double2* in, double2* out,
                 double mass, double r, int dagger, cudaStream_t st);
int wilson_apply_f64(const Geom& g, const double2* U, const double2* in, double2* out,
                     double mass, double r, int dagger, cudaStream_t st);
int sw_cgne(const Geom& g, const SolveArgs& a);
// The inner-precision operators of the mixed modes, through the CG iteration kernels.
int sw_inner_apply(const Geom& g, const double2* U, const double2* W, const double2* in, double2* out, int nsys,
                   const double* masses, double r, int dagger, int precision, cudaStream_t st);
int wilson_inner_apply(const Geom& g, const double2* U, const double2* in, double2* out, int nsys,
                       const double* masses, double r, int dagger, int precision, cudaStream_t st);
int wilson_cgne(const Geom& g, const SolveArgs& a);
// Wilson CGNE on the even-odd Schur complement (FP64 or FP32 inner), solution on the full lattice.
int wilson_cgne_eo(const Geom& g, const SolveArgs& a);

// Tunables set through the C ABI (api.cu), also used by the autotuner.
extern "C" int sw_set_param(int key, double value);
extern "C" int sw_get_param(int key, double* value);

// Argument checks shared by the entry points (api.cu).
int make_geom(const sw_lattice* lat, Geom* g);
int check_buf(const void* p, size_t bytes);
bool overlap(const void* a, size_t na, const void* b, size_t nb);

// Device properties cached per device.
int sm_count();

// Stream-ordered memory pool of the library's device workspace on the current
// device (nullptr if it cannot be created).  Its release threshold keeps
// freed blocks for the next call instead of handing them back to the driver
// at every synchronisation, so a solve does not map gigabytes of workspace
// anew; sw_trim_workspace() returns them.
cudaMemPool_t lib_pool();

// Kernel timing (instrumentation, off by default).  The driver brackets
// sampled launches with events from a pool; once the solve has synchronised,
// prof_flush() turns them into per-class launch counts, times and the
// algorithmic bytes those launches moved.
bool prof_enabled();
cudaEvent_t prof_event();
void prof_push(const char* cls, cudaEvent_t a, cudaEvent_t b, double bytes, double flops = 0.0);
void prof_flush();
// Keep (or drop) the samples pushed since the last commit.
void prof_commit(bool keep);
// Count n launches of a class as issued (while profiling is enabled).
void prof_count(const char* cls, long long n);
// Kernel launches issued by the library (all entry points), for the caller's accounting.
void note_launches(int k);
// Record the CUDA error behind an SW_ERR_CUDA return (sw_last_cuda_error).
int cuda_fail(cudaError_t e);

}  // namespace swc
