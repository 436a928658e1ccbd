// Autotuners for the layout of the inner-precision stencils.
//
// For one operator, precision, lattice and batch size they run the batched
// solve for a fixed number of iterations (the tolerance is unreachable, so
// every candidate does the same work: admission, reliable updates,
// SW_PARAM_CHUNK-sized chunks of CG iterations) with each candidate and keep
// the fastest: sw_autotune over the register-blocking width NS in {1, 2, 4}
// (SW_PARAM_NS_SW or SW_PARAM_NS_WILSON), sw_autotune_layout over width x site
// order (SW_PARAM_SITE_BLOCKING: lexicographic or one of the site-block shapes).
#include <chrono>
#include <vector>

#include "driver.cuh"

namespace swc {

// Deterministic pseudo-random fill in [-1, 1) (a splitmix64 hash of the index).
static __global__ void fill_hash(double2* p, size_t n, unsigned long long seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double a = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    const double b = (double)((z >> 3) & 0xFFFFF) * (1.0 / 1048576.0);
    p[i] = make_double2(2.0 * a - 1.0, 2.0 * b - 1.0);
  }
}

}  // namespace swc

using namespace swc;

namespace {

// Best of two timed batched solves of `iters` iterations each (the tolerance
// is unreachable, so every candidate does the same work), in ms; negative
// SW_ERR_* code on failure.
double time_batch(const Geom& g, int op, const void* U, const void* W, int nsys, int precision, double r,
                  int iters, const std::vector<double>& masses, DevMem& chi, DevMem& x, size_t n, cudaStream_t st) {
  double tmin = 1e300;
  for (int rep = 0; rep < 2; ++rep) {
    cudaMemsetAsync(x.p, 0, sizeof(double2) * n, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SW_ERR_CUDA;
    const auto t0 = std::chrono::steady_clock::now();
    SolveArgs a{static_cast<const double2*>(U), static_cast<const double2*>(W), chi.as<double2>(),
                x.as<double2>(), nsys, masses.data(), r, 1e-30, iters, precision, nullptr, st};
    const int rc = op == SW_OP_WILSON ? wilson_cgne(g, a) : sw_cgne(g, a);
    const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc < 0) return rc;
    if (t < tmin) tmin = t;
  }
  return tmin;
}

// Argument checks and the synthetic batch shared by the autotuners.
int tune_setup(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, int precision, double r,
               int iters, Geom* g, DevMem& chi, DevMem& x, std::vector<double>& masses, size_t* n,
               cudaStream_t st) {
  if (int e = make_geom(lat, g)) return e;
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON) return SW_ERR_ARG;
  if (precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE) return SW_ERR_ARG;
  if (nsys < 1 || nsys > 65535 || iters < 1 || !(r == r)) return SW_ERR_ARG;
  if (int e = check_buf(U, (size_t)g->V * 576)) return e;
  if (op == SW_OP_STAGGERED_WILSON)
    if (int e = check_buf(W, (size_t)g->V * 1152)) return e;
  const int nc = op == SW_OP_WILSON ? 12 : 3;
  *n = (size_t)g->V * nc * nsys;
  if (!chi.alloc(sizeof(double2) * *n, st) || !x.alloc(sizeof(double2) * *n, st)) return SW_ERR_OOM;
  fill_hash<<<sm_count() * 4, 256, 0, st>>>(chi.as<double2>(), *n, 12345ull);
  note_launches(1);
  masses.resize(nsys);
  for (int i = 0; i < nsys; ++i) masses[i] = 0.05 + 0.1 * (i % 4) / 4.0;
  return SW_OK;
}

const int kWidths[3] = {1, 2, 4};
static_assert(kSiteShapes == SW_SITE_SHAPES, "site-shape menu of the C ABI");

}  // namespace

extern "C" int sw_autotune(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, int precision,
                           double r, int iters, double* ms, int* best, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Geom g;
  DevMem chi, x;
  std::vector<double> masses;
  size_t n = 0;
  if (int e = tune_setup(lat, op, U, W, nsys, precision, r, iters, &g, chi, x, masses, &n, st)) return e;
  const int key = op == SW_OP_WILSON ? SW_PARAM_NS_WILSON : SW_PARAM_NS_SW;
  double keep = 0;
  sw_get_param(key, &keep);
  double best_ms = 1e300;
  int best_ns = (int)keep;
  for (int k = 0; k < 3; ++k) {
    sw_set_param(key, kWidths[k]);
    const double t = time_batch(g, op, U, W, nsys, precision, r, iters, masses, chi, x, n, st);
    if (t < 0) {
      sw_set_param(key, keep);
      return (int)t;
    }
    if (ms) ms[k] = t;
    if (t < best_ms) {
      best_ms = t;
      best_ns = kWidths[k];
    }
  }
  sw_set_param(key, best_ns);
  if (best) *best = best_ns;
  return SW_OK;
}

extern "C" int sw_autotune_layout(const sw_lattice* lat, int op, const void* U, const void* W, int nsys,
                                  int precision, double r, int iters, double* ms, int* best_ns,
                                  int* best_shape, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Geom g;
  DevMem chi, x;
  std::vector<double> masses;
  size_t n = 0;
  if (int e = tune_setup(lat, op, U, W, nsys, precision, r, iters, &g, chi, x, masses, &n, st)) return e;
  const int key = op == SW_OP_WILSON ? SW_PARAM_NS_WILSON : SW_PARAM_NS_SW;
  double keep_ns = 0, keep_shape = 0;
  sw_get_param(key, &keep_ns);
  sw_get_param(SW_PARAM_SITE_BLOCKING, &keep_shape);
  double best_ms = 1e300;
  int bns = (int)keep_ns, bshape = (int)keep_shape;
  for (int k = 0; k < 3; ++k)
    for (int shape = 0; shape < SW_SITE_SHAPES; ++shape) {
      sw_set_param(key, kWidths[k]);
      Geom gs = g;  // the candidate's site order (a solve takes it from its Geom)
      gs.shape = shape;
      const double t = time_batch(gs, op, U, W, nsys, precision, r, iters, masses, chi, x, n, st);
      if (t < 0) {
        sw_set_param(key, keep_ns);
        return (int)t;
      }
      if (ms) ms[k * SW_SITE_SHAPES + shape] = t;
      if (t < best_ms) {
        best_ms = t;
        bns = kWidths[k];
        bshape = shape;
      }
    }
  sw_set_param(key, bns);
  sw_set_param(SW_PARAM_SITE_BLOCKING, bshape);
  if (best_ns) *best_ns = bns;
  if (best_shape) *best_shape = bshape;
  return SW_OK;
}
