// C ABI entry points (include/sw_cgne.h): argument checks, then dispatch.
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace swc {


cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cached[dev] = n;
  }
  return cached[dev];
}

// ---------------------------------------------------------------- profiler
namespace {
struct ProfStat {
  long long launches = 0;
  long long issued = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double flops = 0.0;
};
struct Pending {
  std::string cls;
  cudaEvent_t a, b;
  double bytes, flops;
};
std::mutex g_prof_mu;
std::atomic<long long> g_launches{0};
bool g_prof_on = false;
std::map<std::string, ProfStat> g_prof;
std::vector<cudaEvent_t> g_pool;
thread_local std::vector<Pending> t_pending;
thread_local std::vector<Pending> t_staged;
std::atomic<int> g_param_chunk{4};
std::atomic<double> g_param_delta{3e-5};
std::atomic<double> g_param_delta16{1e-3};
std::atomic<int> g_param_ns_sw{2};
std::atomic<int> g_param_ns_wilson{1};
std::atomic<int> g_param_graphs{1};
std::atomic<int> g_param_persistent{0};
std::atomic<int> g_param_wilson_lean{-1};
std::atomic<int> g_param_site_block{0};
std::atomic<int> g_param_group_fast{0};
thread_local std::vector<cudaEvent_t> t_used;
}  // namespace

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

std::atomic<int> g_last_cuda_error{0};
int cuda_fail(cudaError_t e) {
  g_last_cuda_error.store((int)e);
  return SW_ERR_CUDA;
}

bool prof_enabled() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof_on;
}

cudaEvent_t prof_event() {
  cudaEvent_t e = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_pool.empty()) {
      e = g_pool.back();
      g_pool.pop_back();
    }
  }
  if (!e) cudaEventCreate(&e);
  t_used.push_back(e);
  return e;
}

void prof_push(const char* cls, cudaEvent_t a, cudaEvent_t b, double bytes, double flops) {
  t_staged.push_back(Pending{cls, a, b, bytes, flops});
}

void prof_count(const char* cls, long long n) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_on) g_prof[cls].issued += n;
}

void prof_commit(bool keep) {
  if (keep) t_pending.insert(t_pending.end(), t_staged.begin(), t_staged.end());
  t_staged.clear();
}

int param_chunk() { return g_param_chunk.load(); }
double param_delta(bool half) { return half ? g_param_delta16.load() : g_param_delta.load(); }
int param_ns(int nc) { return nc == 3 ? g_param_ns_sw.load() : g_param_ns_wilson.load(); }
bool param_graphs() { return g_param_graphs.load() != 0; }
bool param_persistent() { return g_param_persistent.load() != 0; }
int param_wilson_lean() { return g_param_wilson_lean.load(); }
int param_site_shape() { return g_param_site_block.load(); }
bool param_group_fast() { return g_param_group_fast.load() != 0; }

void prof_flush() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const Pending& p : t_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ProfStat& s = g_prof[p.cls];
      s.launches += 1;
      s.ms += ms;
      s.bytes += p.bytes;
      s.flops += p.flops;
    } else {
      cudaGetLastError();
    }
  }
  t_pending.clear();
  t_staged.clear();
  for (cudaEvent_t e : t_used) g_pool.push_back(e);
  t_used.clear();
}

int make_geom(const sw_lattice* lat, Geom* g) {
  if (!lat) return SW_ERR_NULL;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int L = lat->dims[mu];
    if (L < 2 || (L & 1)) return SW_ERR_DIMS;
    V *= L;
    if (V > (1LL << 28)) return SW_ERR_DIMS;
  }
  for (int mu = 0; mu < 4; ++mu) g->L[mu] = lat->dims[mu];
  g->stride[0] = 1;
  for (int mu = 1; mu < 4; ++mu) g->stride[mu] = g->stride[mu - 1] * g->L[mu - 1];
  g->V = (int)V;
  g->apbc = lat->t_antiperiodic ? 1 : 0;
  g->shape = param_site_shape();
  return SW_OK;
}

// Driver entry point for the allocation extent of a device pointer.
typedef int (*AddrRangeFn)(unsigned long long*, size_t*, unsigned long long);
static AddrRangeFn addr_range_fn() {
  static std::once_flag once;
  static AddrRangeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<AddrRangeFn>(p);
  });
  return fn;
}

// The buffer must be device (or managed) memory, 16-byte aligned, and its
// allocation must hold `bytes` from `p` on.
int check_buf(const void* p, size_t bytes) {
  if (!p) return SW_ERR_NULL;
  if (reinterpret_cast<uintptr_t>(p) & 15u) return SW_ERR_ALIGN;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return SW_ERR_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return SW_ERR_ARG;
  if (AddrRangeFn fn = addr_range_fn()) {
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, reinterpret_cast<unsigned long long>(p)) != 0) return SW_ERR_ARG;
    if (reinterpret_cast<unsigned long long>(p) + bytes > base + size) return SW_ERR_ARG;
  }
  return SW_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

#define SW_TRY(expr)            \
  do {                          \
    const int _e = (expr);      \
    if (_e != SW_OK) return _e; \
  } while (0)

}  // namespace swc

using namespace swc;

extern "C" {

const char* sw_last_cuda_error(void) { return cudaGetErrorName((cudaError_t)g_last_cuda_error.load()); }

const char* sw_status_string(int s) {
  switch (s) {
    case SW_OK: return "ok";
    case SW_NOT_CONVERGED: return "not converged (max_iter reached)";
    case SW_ERR_DIMS: return "bad lattice extents (each must be even and >= 2)";
    case SW_ERR_NULL: return "null pointer argument";
    case SW_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case SW_ERR_CUDA: return "CUDA error";
    case SW_ERR_NAN: return "non-finite residual or CG breakdown";
    case SW_ERR_OOM: return "device workspace allocation failed";
    case SW_ERR_TIMEOUT: return "bounded wait gave up";
    case SW_ERR_ARG: return "bad argument";
    default: return "unknown status";
  }
}

int sw_set_param(int key, double value) {
  switch (key) {
    case SW_PARAM_CHUNK:
      if (!(value >= 1 && value <= 4096)) return SW_ERR_ARG;
      g_param_chunk.store((int)value);
      return SW_OK;
    case SW_PARAM_RELIABLE_DELTA:
    case SW_PARAM_RELIABLE_DELTA_F16:
      if (!(value > 0 && value < 1)) return SW_ERR_ARG;
      (key == SW_PARAM_RELIABLE_DELTA ? g_param_delta : g_param_delta16).store(value);
      return SW_OK;
    case SW_PARAM_GRAPHS:
    case SW_PARAM_GROUP_FAST:
    case SW_PARAM_PERSISTENT:
      if (!(value == 0 || value == 1)) return SW_ERR_ARG;
      (key == SW_PARAM_GRAPHS ? g_param_graphs : key == SW_PARAM_GROUP_FAST ? g_param_group_fast
                                                                               : g_param_persistent)
          .store((int)value);
      return SW_OK;
    case SW_PARAM_WILSON_LEAN:
      if (!(value == -1 || value == 0 || value == 1)) return SW_ERR_ARG;
      g_param_wilson_lean.store((int)value);
      return SW_OK;
    case SW_PARAM_SITE_BLOCKING:
      if (!(value >= 0 && value < SW_SITE_SHAPES && value == (int)value)) return SW_ERR_ARG;
      g_param_site_block.store((int)value);
      return SW_OK;
    case SW_PARAM_NS_SW:
    case SW_PARAM_NS_WILSON:
      if (!(value == 1 || value == 2 || value == 4)) return SW_ERR_ARG;
      (key == SW_PARAM_NS_SW ? g_param_ns_sw : g_param_ns_wilson).store((int)value);
      return SW_OK;
    default:
      return SW_ERR_ARG;
  }
}

int sw_get_param(int key, double* value) {
  if (!value) return SW_ERR_NULL;
  switch (key) {
    case SW_PARAM_CHUNK: *value = g_param_chunk.load(); return SW_OK;
    case SW_PARAM_RELIABLE_DELTA: *value = g_param_delta.load(); return SW_OK;
    case SW_PARAM_RELIABLE_DELTA_F16: *value = g_param_delta16.load(); return SW_OK;
    case SW_PARAM_NS_SW: *value = g_param_ns_sw.load(); return SW_OK;
    case SW_PARAM_NS_WILSON: *value = g_param_ns_wilson.load(); return SW_OK;
    case SW_PARAM_GRAPHS: *value = g_param_graphs.load(); return SW_OK;
    case SW_PARAM_SITE_BLOCKING: *value = g_param_site_block.load(); return SW_OK;
    case SW_PARAM_GROUP_FAST: *value = g_param_group_fast.load(); return SW_OK;
    case SW_PARAM_PERSISTENT: *value = g_param_persistent.load(); return SW_OK;
    case SW_PARAM_WILSON_LEAN: *value = g_param_wilson_lean.load(); return SW_OK;
    default: return SW_ERR_ARG;
  }
}

long long sw_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int sw_trim_workspace(void) {
  cudaMemPool_t pool = lib_pool();
  if (!pool) return SW_ERR_CUDA;
  if (const cudaError_t e = cudaMemPoolTrimTo(pool, 0); e != cudaSuccess) return cuda_fail(e);
  return SW_OK;
}

int sw_workspace_reserved(unsigned long long* bytes) {
  if (!bytes) return SW_ERR_NULL;
  cudaMemPool_t pool = lib_pool();
  if (!pool) return SW_ERR_CUDA;
  unsigned long long v = 0;
  if (const cudaError_t e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v); e != cudaSuccess)
    return cuda_fail(e);
  *bytes = (unsigned long long)v;
  return SW_OK;
}

int sw_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return SW_OK;
}

int sw_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.clear();
  return SW_OK;
}

int sw_profile_issued(int i, long long* issued) {
  if (!issued) return SW_ERR_NULL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (i < 0 || i >= (int)g_prof.size()) return SW_ERR_ARG;
  auto it = g_prof.begin();
  std::advance(it, i);
  *issued = it->second.issued;
  return SW_OK;
}

int sw_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return (int)g_prof.size();
}

int sw_profile_entry(int i, char* name, int name_len, long long* launches, double* total_ms,
                     double* total_bytes, double* total_flops) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (i < 0 || i >= (int)g_prof.size()) return SW_ERR_ARG;
  auto it = g_prof.begin();
  std::advance(it, i);
  if (name && name_len > 0) {
    std::strncpy(name, it->first.c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = it->second.launches;
  if (total_ms) *total_ms = it->second.ms;
  if (total_bytes) *total_bytes = it->second.bytes;
  if (total_flops) *total_flops = it->second.flops;
  return SW_OK;
}

int sw_hypercube_build(const sw_lattice* lat, const void* U, void* W, void* stream) {
  Geom g;
  SW_TRY(make_geom(lat, &g));
  const size_t V = g.V;
  SW_TRY(check_buf(U, V * 4 * 9 * 16));
  SW_TRY(check_buf(W, V * 8 * 9 * 16));
  if (overlap(U, V * 576, W, V * 1152)) return SW_ERR_ARG;
  return hypercube_build_f64(g, static_cast<const double2*>(U), static_cast<double2*>(W),
                             static_cast<cudaStream_t>(stream));
}

int sw_dslash_apply(const sw_lattice* lat, const void* U, const void* W, const void* in, void* out, double mass,
                    double r, int dagger, void* stream) {
  Geom g;
  SW_TRY(make_geom(lat, &g));
  const size_t V = g.V;
  SW_TRY(check_buf(U, V * 576));
  SW_TRY(check_buf(W, V * 1152));
  SW_TRY(check_buf(in, V * 48));
  SW_TRY(check_buf(out, V * 48));
  if (overlap(in, V * 48, out, V * 48)) return SW_ERR_ARG;
  return sw_apply_f64(g, static_cast<const double2*>(U), static_cast<const double2*>(W),
                      static_cast<const double2*>(in), static_cast<double2*>(out), mass, r, dagger,
                      static_cast<cudaStream_t>(stream));
}

int wilson_dslash_apply(const sw_lattice* lat, const void* U, const void* in, void* out, double mass, double r,
                        int dagger, void* stream) {
  Geom g;
  SW_TRY(make_geom(lat, &g));
  const size_t V = g.V;
  SW_TRY(check_buf(U, V * 576));
  SW_TRY(check_buf(in, V * 192));
  SW_TRY(check_buf(out, V * 192));
  if (overlap(in, V * 192, out, V * 192)) return SW_ERR_ARG;
  return wilson_apply_f64(g, static_cast<const double2*>(U), static_cast<const double2*>(in),
                          static_cast<double2*>(out), mass, r, dagger, static_cast<cudaStream_t>(stream));
}

int cgne_solve(const sw_lattice* lat, int op, const void* U, const void* W, const void* chi, void* x, double mass,
               double r, double tol, int max_iter, int precision, sw_solve_info* info, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) *info = sw_solve_info{};
  Geom g;
  SW_TRY(make_geom(lat, &g));
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON && op != SW_OP_WILSON_EVEN_ODD) return SW_ERR_ARG;
  if (precision != SW_PREC_F64 && precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE)
    return SW_ERR_ARG;
  if (op == SW_OP_WILSON_EVEN_ODD && precision == SW_PREC_F16_RELIABLE) return SW_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0) || max_iter < 1) return SW_ERR_ARG;
  if (!(mass == mass) || !(r == r)) return SW_ERR_ARG;
  const size_t V = g.V;
  const size_t vb = V * (op != SW_OP_STAGGERED_WILSON ? 192 : 48);
  SW_TRY(check_buf(U, V * 576));
  if (op == SW_OP_STAGGERED_WILSON) SW_TRY(check_buf(W, V * 1152));
  SW_TRY(check_buf(chi, vb));
  SW_TRY(check_buf(x, vb));
  if (overlap(chi, vb, x, vb)) return SW_ERR_ARG;
  SolveArgs a{static_cast<const double2*>(U), static_cast<const double2*>(W), static_cast<const double2*>(chi),
              static_cast<double2*>(x), 1, &mass, r, tol, max_iter, precision, info,
              static_cast<cudaStream_t>(stream)};
  const int rc = (op == SW_OP_WILSON) ? wilson_cgne(g, a) : (op == SW_OP_WILSON_EVEN_ODD) ? wilson_cgne_eo(g, a)
                                                                                           : sw_cgne(g, a);
  if (info) {
    info->status = rc;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int cgne_solve_batch(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, const void* chi,
                     void* x, const double* masses, double r, double tol, int max_iter, int precision,
                     sw_solve_info* infos, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (nsys < 1 || nsys > 65535) return SW_ERR_ARG;
  if (!masses) return SW_ERR_NULL;
  if (infos)
    for (int i = 0; i < nsys; ++i) infos[i] = sw_solve_info{};
  Geom g;
  SW_TRY(make_geom(lat, &g));
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON && op != SW_OP_WILSON_EVEN_ODD) return SW_ERR_ARG;
  if (precision != SW_PREC_F64 && precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE)
    return SW_ERR_ARG;
  if (op == SW_OP_WILSON_EVEN_ODD && precision == SW_PREC_F16_RELIABLE) return SW_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0) || max_iter < 1) return SW_ERR_ARG;
  for (int i = 0; i < nsys; ++i)
    if (!(masses[i] == masses[i])) return SW_ERR_ARG;
  if (!(r == r)) return SW_ERR_ARG;
  const size_t V = g.V;
  const size_t vb = V * (op != SW_OP_STAGGERED_WILSON ? 192 : 48) * (size_t)nsys;
  SW_TRY(check_buf(U, V * 576));
  if (op == SW_OP_STAGGERED_WILSON) SW_TRY(check_buf(W, V * 1152));
  SW_TRY(check_buf(chi, vb));
  SW_TRY(check_buf(x, vb));
  if (overlap(chi, vb, x, vb)) return SW_ERR_ARG;
  SolveArgs a{static_cast<const double2*>(U), static_cast<const double2*>(W), static_cast<const double2*>(chi),
              static_cast<double2*>(x), nsys, masses, r, tol, max_iter, precision, infos,
              static_cast<cudaStream_t>(stream)};
  const int rc = (op == SW_OP_WILSON) ? wilson_cgne(g, a) : (op == SW_OP_WILSON_EVEN_ODD) ? wilson_cgne_eo(g, a)
                                                                                           : sw_cgne(g, a);
  if (infos) {
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < nsys; ++i) infos[i].seconds = secs;
  }
  return rc;
}


int dslash_apply_inner(const sw_lattice* lat, int op, const void* U, const void* W, int nsys, const void* in,
                       void* out, const double* masses, double r, int dagger, int precision, void* stream) {
  Geom g;
  SW_TRY(make_geom(lat, &g));
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON) return SW_ERR_ARG;
  if (precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE) return SW_ERR_ARG;
  if (nsys < 1 || nsys > 65535) return SW_ERR_ARG;
  if (!masses) return SW_ERR_NULL;
  for (int i = 0; i < nsys; ++i)
    if (!(masses[i] == masses[i])) return SW_ERR_ARG;
  if (!(r == r)) return SW_ERR_ARG;
  const size_t V = g.V;
  const size_t vb = V * (op == SW_OP_WILSON ? 192 : 48) * (size_t)nsys;
  SW_TRY(check_buf(U, V * 576));
  if (op == SW_OP_STAGGERED_WILSON) SW_TRY(check_buf(W, V * 1152));
  SW_TRY(check_buf(in, vb));
  SW_TRY(check_buf(out, vb));
  if (overlap(in, vb, out, vb)) return SW_ERR_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const auto* u = static_cast<const double2*>(U);
  const auto* v = static_cast<const double2*>(in);
  auto* o = static_cast<double2*>(out);
  return (op == SW_OP_WILSON)
             ? wilson_inner_apply(g, u, v, o, nsys, masses, r, dagger, precision, st)
             : sw_inner_apply(g, u, static_cast<const double2*>(W), v, o, nsys, masses, r, dagger, precision, st);
}

}  // extern "C"
