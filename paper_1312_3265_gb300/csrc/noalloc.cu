// cgne_solve_noalloc: the FP64 CGNE solve with its device workspace in a
// fixed, file-scope device array instead of memory allocated per call.
//
// For callers that cannot call cudaMalloc (or any other allocator) while they
// run: plugins and host runtimes whose device memory is owned and budgeted by
// another allocator, so that an allocation behind its back would break its
// accounting or fail, and latency-critical loops that must never enter the
// driver's allocator.  They pass their inputs and outputs; the library
// supplies the scratch.  The call also creates no stream, event or graph, and
// it blocks until the solve is done (it reads the solver's status words on the
// host between rounds of iterations).
//
// The scratch array (kNoallocScratchBytes) is part of the module, so every
// GPU that loads the library holds it until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress, on the
// first call made with that device current.  All calls share the one array
// and it keeps the previous call's contents: everything the solve reads is
// initialised by the solve itself.  No two calls may be in progress at the
// same time -- on one stream or several, from one host thread or several --
// because each would overwrite the other's vectors and status words; the
// caller serialises them.
#include <mutex>

#include "driver.cuh"

namespace swc {

constexpr size_t kNoallocScratchBytes = 32ull << 20;  // SW_NOALLOC_SCRATCH_BYTES

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

using SWd = SWOp<double, GaugeC64, TransC64, VecC64>;
template <bool R1> using Wd = WOp<double, GaugeC64, VecC64, R1>;

// Device address of the scratch array for the current device (set up once per
// device); nullptr if the lookup fails.
static void* noalloc_scratch() {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace swc

using namespace swc;

extern "C" int cgne_solve_noalloc(const sw_lattice* lat, int op, const void* U, const void* W, const void* chi,
                                  void* x, double mass, double r, double tol, int max_iter, sw_solve_info* info,
                                  void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (info) *info = sw_solve_info{};
  Geom g;
  if (int e = make_geom(lat, &g)) return e;
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON) return SW_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0) || max_iter < 1) return SW_ERR_ARG;
  if (!(mass == mass) || !(r == r)) return SW_ERR_ARG;
  const int NC = (op == SW_OP_WILSON) ? 12 : 3;
  if (workspace_bytes(g.V, NC, 1, false) > kNoallocScratchBytes) return SW_ERR_ARG;
  const size_t V = g.V;
  const size_t vb = V * NC * 16;
  if (int e = check_buf(U, V * 576)) return e;
  if (op == SW_OP_STAGGERED_WILSON)
    if (int e = check_buf(W, V * 1152)) return e;
  if (int e = check_buf(chi, vb)) return e;
  if (int e = check_buf(x, vb)) return e;
  if (overlap(chi, vb, x, vb)) return SW_ERR_ARG;
  void* scratch = noalloc_scratch();
  if (!scratch) return SW_ERR_CUDA;

  SolveArgs a{static_cast<const double2*>(U), static_cast<const double2*>(W), static_cast<const double2*>(chi),
              static_cast<double2*>(x), 1, &mass, r, tol, max_iter, SW_PREC_F64, info,
              static_cast<cudaStream_t>(stream)};
  const Workspace ws = carve_workspace(scratch, g.V, NC, 1, false);
  SysState hs[2];  // status words travel through ordinary host memory
  int rc;
  if (op == SW_OP_STAGGERED_WILSON) {
    const SWd opd{GaugeC64{a.U}, TransC64{a.W}};
    rc = run_cgne_ws<SWd, SWd, false>(g, opd, opd, a, ws, hs, false);
  } else if (r == 1.0) {
    const Wd<true> opd{GaugeC64{a.U}};
    rc = run_cgne_ws<Wd<true>, Wd<true>, false>(g, opd, opd, a, ws, hs, false);
  } else {
    const Wd<false> opd{GaugeC64{a.U}};
    rc = run_cgne_ws<Wd<false>, Wd<false>, false>(g, opd, opd, a, ws, hs, false);
  }
  if (info) {
    info->status = rc;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}
