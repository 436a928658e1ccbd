// Host driver of the batched CGNE solve (Eq. 2), shared by both operators.
//
// Precision modes
//   F64    x, r, p, t in FP64 (canonical layout); the residual is replaced by
//          the recomputed b - A x whenever the iterated one meets the
//          tolerance, so convergence is always decided on a true residual.
//   MIXED  inner iterations in FP32 on planar copies of links and vectors,
//          with reliable updates (Sleijpen & van der Vorst 1996): when the
//          iterated residual falls below delta times its maximum since the
//          last update (or meets the tolerance), the FP32 correction is
//          added to the FP64 solution and r = b - A x is recomputed in FP64.
//          Dot products always accumulate in FP64.
//
// The host launches iterations in chunks and reads the per-system status
// words between chunks; iterations of systems that have stopped return at
// once on the device.
#pragma once
#include <chrono>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "misc_kernels.cuh"

namespace swc {

constexpr int kChunk = 16;
constexpr double kReliableDelta = 0.1;

inline int grid_for(const void* kernel, int block, int V, int nsys, int cap) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  int nb;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(kernel);
    if (it == cache.end()) {
      nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess || nb < 1) nb = 1;
      cache[kernel] = nb;
    } else {
      nb = it->second;
    }
  }
  int gx = (sm_count() * nb) / (nsys > 0 ? nsys : 1);
  if (gx < 1) gx = 1;
  const int need = (V + block - 1) / block;
  if (gx > need) gx = need;
  if (gx > cap) gx = cap;
  return gx;
}

// Stream-ordered device allocation, freed on scope exit.
struct DevMem {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() {
    if (p) cudaFreeAsync(p, s);
  }
  bool alloc(size_t bytes, cudaStream_t st) {
    s = st;
    return cudaMallocAsync(&p, bytes ? bytes : 16, st) == cudaSuccess;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

inline int pinned_states(int nsys, SysState** out) {
  thread_local SysState* buf = nullptr;
  thread_local int cap = 0;
  if (nsys > cap) {
    if (buf) cudaFreeHost(buf);
    buf = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&buf, sizeof(SysState) * nsys) != cudaSuccess) return SW_ERR_OOM;
    cap = nsys;
  }
  *out = buf;
  return SW_OK;
}

inline int status_to_code(int st) {
  switch (st) {
    case ST_CONVERGED: return SW_OK;
    case ST_MAXITER: return SW_NOT_CONVERGED;
    case ST_FAILED: return SW_ERR_NAN;
    default: return SW_ERR_TIMEOUT;
  }
}

// Device workspace of one batched solve, carved from a single block.
struct Workspace {
  double2 *b64, *r64, *t64, *p64;   // FP64 canonical; p64 only in F64 mode
  float2 *r32, *p32, *t32, *x32;    // FP32 planar; MIXED mode only
  SysState* S;
  double* partials;
  unsigned* tickets;
  double* mass;
};

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Bytes of workspace for nsys systems of NC complex components per site.
inline size_t workspace_bytes(int V, int NC, int nsys, bool mixed) {
  const size_t n = (size_t)V * NC * nsys;
  const size_t ntiles = (size_t)(V + kTile - 1) / kTile;
  size_t b = 3 * align_up(sizeof(double2) * n);
  b += mixed ? 4 * align_up(sizeof(float2) * n) : align_up(sizeof(double2) * n);
  b += align_up(sizeof(SysState) * nsys) + align_up(sizeof(double) * ntiles * nsys) +
       align_up(sizeof(unsigned) * nsys) + align_up(sizeof(double) * nsys);
  return b;
}

inline Workspace carve_workspace(void* base, int V, int NC, int nsys, bool mixed) {
  const size_t n = (size_t)V * NC * nsys;
  const size_t ntiles = (size_t)(V + kTile - 1) / kTile;
  char* c = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    void* p = c;
    c += align_up(bytes);
    return p;
  };
  Workspace w{};
  w.b64 = (double2*)take(sizeof(double2) * n);
  w.r64 = (double2*)take(sizeof(double2) * n);
  w.t64 = (double2*)take(sizeof(double2) * n);
  if (mixed) {
    w.r32 = (float2*)take(sizeof(float2) * n);
    w.p32 = (float2*)take(sizeof(float2) * n);
    w.t32 = (float2*)take(sizeof(float2) * n);
    w.x32 = (float2*)take(sizeof(float2) * n);
  } else {
    w.p64 = (double2*)take(sizeof(double2) * n);
  }
  w.S = (SysState*)take(sizeof(SysState) * nsys);
  w.partials = (double*)take(sizeof(double) * ntiles * nsys);
  w.tickets = (unsigned*)take(sizeof(unsigned) * nsys);
  w.mass = (double*)take(sizeof(double) * nsys);
  return w;
}

// OpD: FP64 operator on canonical storage.  OpF: the inner-iteration operator
// (FP32 planar when MIXED, else the same as OpD).  ws: device workspace from
// carve_workspace; hs: host array [nsys] for the status words.
template <class OpD, class OpF, bool MIXED>
int run_cgne_ws(const Geom& g, const OpD& opd, const OpF& opf, const SolveArgs& a, const Workspace& ws,
                SysState* hs) {
  using namespace std::chrono;
  const auto t0 = steady_clock::now();
  constexpr int NC = OpD::NC;
  using V64 = typename OpD::Vec;
  using VF = typename OpF::Vec;
  using TF = typename std::conditional<MIXED, float, double>::type;
  const int nsys = a.nsys;
  const int V = g.V;
  const size_t n = (size_t)V * NC;
  cudaStream_t st = a.stream;
  const int pstride = (V + kTile - 1) / kTile;  // one partial per reduction tile

  double2* b64 = ws.b64;
  double2* r64 = ws.r64;
  double2* t64 = ws.t64;
  SysState* S = ws.S;
  RedBuf rb{ws.partials, ws.tickets, pstride};
  double* mass_d = ws.mass;

  for (int i = 0; i < nsys; ++i) {
    SysState s{};
    s.tol2 = a.tol * a.tol;
    s.delta2 = MIXED ? kReliableDelta * kReliableDelta : 0.0;
    s.max_iter = a.max_iter;
    s.status = ST_NEED_RU;
    hs[i] = s;
  }
  cudaMemcpyAsync(S, hs, sizeof(SysState) * nsys, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(mass_d, a.masses, sizeof(double) * nsys, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(rb.tickets, 0, sizeof(unsigned) * nsys, st);

  V64 chi{const_cast<double2*>(a.chi)}, vb{b64}, vr{r64}, vt{t64}, vx{a.x};
  BatchParams bp{mass_d, a.r, n, n};

  const int gA = grid_for((const void*)apply_kernel<double, OpD>, kTile, V, nsys, pstride);
  const int gR = grid_for((const void*)residual64<OpD>, kTile, V, nsys, pstride);
  const int gV = grid_for((const void*)cg_k3<TF, VF, NC>, 256, V, nsys, pstride);
  const int gN = grid_for((const void*)norm_b<NC>, kTile, V, nsys, pstride);
  const int g1 = grid_for((const void*)cg_k1<TF, OpF>, kTile, V, nsys, pstride);
  const int g2 = grid_for((const void*)cg_k2<TF, OpF, VF>, kTile, V, nsys, pstride);

  // b = (D+m)^+ chi, |b|^2
  apply_kernel<double, OpD><<<dim3(gA, nsys), kTile, 0, st>>>(g, opd, chi, vb, 0.0, mass_d, n, a.r, 1, nullptr, 0);
  norm_b<NC><<<dim3(gN, nsys), kTile, 0, st>>>(V, b64, n, S, rb);
  note_launches(2);

  VF fr, fp, ft, fx;
  if constexpr (MIXED) {
    fr = VF{ws.r32, V};
    fp = VF{ws.p32, V};
    ft = VF{ws.t32, V};
    fx = VF{ws.x32, V};
    cudaMemsetAsync(ws.p32, 0, sizeof(float2) * n * nsys, st);
    cudaMemsetAsync(ws.x32, 0, sizeof(float2) * n * nsys, st);
  } else {
    fr = vr;
    fp = VF{ws.p64};
    ft = vt;
    fx = vx;
    cudaMemsetAsync(ws.p64, 0, sizeof(double2) * n * nsys, st);
  }

  // |b| = 0: the solution is x = 0
  cudaMemcpyAsync(hs, S, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return SW_ERR_CUDA;
  bool any_zero = false;
  for (int i = 0; i < nsys; ++i)
    if (hs[i].b2 == 0.0) {
      any_zero = true;
      hs[i].status = ST_CONVERGED;
      hs[i].rr_true = 0.0;
      cudaMemsetAsync(a.x + (size_t)i * n, 0, sizeof(double2) * n, st);
    }
  if (any_zero) cudaMemcpyAsync(S, hs, sizeof(SysState) * nsys, cudaMemcpyHostToDevice, st);

  auto reliable_update = [&]() {
    if constexpr (MIXED)
      accum_x<NC><<<dim3(gV, nsys), 256, 0, st>>>(V, a.x, fx.p, n, n, S);
    apply_kernel<double, OpD><<<dim3(gA, nsys), kTile, 0, st>>>(g, opd, vx, vt, 0.0, mass_d, n, a.r, 0, S, ST_NEED_RU);
    residual64<OpD><<<dim3(gR, nsys), kTile, 0, st>>>(g, opd, vt, vb, vr, bp, S, rb);
    if constexpr (MIXED) demote_r<NC><<<dim3(gV, nsys), 256, 0, st>>>(V, r64, fr.p, n, n, S);
    cg_k3<TF, VF, NC><<<dim3(gV, nsys), 256, 0, st>>>(V, fr, fp, n, S, ST_JUST_UPDATED);
    commit_status<<<(nsys + 127) / 128, 128, 0, st>>>(nsys, S);
    note_launches(MIXED ? 6 : 4);
  };
  // Algorithmic bytes of one stencil launch (every stored element touched
  // once): the links (and transports) once per launch, plus per running
  // system the vectors the kernel reads and writes (k1: p, t; k2: t, p, x and
  // r read and written).
  constexpr double kCx = 2.0 * sizeof(TF);
  const double gauge_bytes = (double)V * OpF::kMats * 9 * kCx;
  const double vec_bytes = (double)V * NC * kCx;
  static const std::string cls1 = std::string(OpF::kName) + (MIXED ? ".k1.f32" : ".k1.f64");
  static const std::string cls2 = std::string(OpF::kName) + (MIXED ? ".k2.f32" : ".k2.f64");
  auto iterate = [&](int nrun) {
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (nrun > 0) {
      e0 = prof_event();
      e1 = prof_event();
      e2 = prof_event();
      cudaEventRecord(e0, st);
    }
    cg_k1<TF, OpF><<<dim3(g1, nsys), kTile, 0, st>>>(g, opf, fp, ft, bp, S, rb);
    if (nrun > 0) cudaEventRecord(e1, st);
    cg_k2<TF, OpF, VF><<<dim3(g2, nsys), kTile, 0, st>>>(g, opf, ft, fp, fr, fx, bp, n, S, rb);
    if (nrun > 0) {
      cudaEventRecord(e2, st);
      prof_push(cls1.c_str(), e0, e1, gauge_bytes + nrun * 2.0 * vec_bytes);
      prof_push(cls2.c_str(), e1, e2, gauge_bytes + nrun * 6.0 * vec_bytes);
    }
    cg_k3<TF, VF, NC><<<dim3(gV, nsys), 256, 0, st>>>(V, fr, fp, n, S, ST_RUNNING);
    note_launches(3);
  };

  // initial residual r = b - A x0 (all systems start in NEED_RU)
  reliable_update();
  const long long max_rounds = 4LL * (a.max_iter / kChunk + 2) + 1000;
  int rc = SW_OK;
  for (long long round = 0;; ++round) {
    cudaMemcpyAsync(hs, S, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SW_ERR_CUDA;
    bool need_ru = false, active = false;
    int nrun = 0;
    for (int i = 0; i < nsys; ++i) {
      const int s = hs[i].status;
      need_ru |= (s == ST_NEED_RU);
      active |= (s == ST_RUNNING || s == ST_NEED_RU || s == ST_JUST_UPDATED);
      nrun += (s == ST_RUNNING);
    }
    if (!active) break;
    if (round > max_rounds) {
      rc = SW_ERR_TIMEOUT;
      break;
    }
    if (need_ru) {
      reliable_update();
      continue;
    }
    const bool prof = prof_enabled();
    for (int i = 0; i < kChunk; ++i) iterate((prof && i == 0) ? nrun : 0);
    if (cudaPeekAtLastError() != cudaSuccess) return SW_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return SW_ERR_CUDA;
  prof_flush();

  const double secs = duration<double>(steady_clock::now() - t0).count();
  int worst = SW_OK;
  for (int i = 0; i < nsys; ++i) {
    const int code = (rc != SW_OK) ? rc : status_to_code(hs[i].status);
    if (a.infos) {
      sw_solve_info& inf = a.infos[i];
      inf.iters = hs[i].iter;
      inf.reliable_updates = hs[i].n_ru;
      inf.status = code;
      inf.precision = a.precision;
      inf.true_rel_resid = hs[i].b2 > 0 ? sqrt(hs[i].rr_true / hs[i].b2) : 0.0;
      inf.seconds = secs;
    }
    if (code < 0 && (worst >= 0 || code < worst)) worst = code;
    if (code > 0 && worst == SW_OK) worst = code;
  }
  return worst;
}

// Allocating entry: one stream-ordered block of workspace for the call and a
// pinned host buffer for the status words.
template <class OpD, class OpF, bool MIXED>
int run_cgne(const Geom& g, const OpD& opd, const OpF& opf, const SolveArgs& a) {
  DevMem mem;
  if (!mem.alloc(workspace_bytes(g.V, OpD::NC, a.nsys, MIXED), a.stream)) return SW_ERR_OOM;
  SysState* hs = nullptr;
  if (int e = pinned_states(a.nsys, &hs)) return e;
  const Workspace ws = carve_workspace(mem.p, g.V, OpD::NC, a.nsys, MIXED);
  return run_cgne_ws<OpD, OpF, MIXED>(g, opd, opf, a, ws, hs);
}

}  // namespace swc
