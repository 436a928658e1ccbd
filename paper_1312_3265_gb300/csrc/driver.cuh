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

// OpD: FP64 operator on canonical storage.  OpF: the inner-iteration operator
// (FP32 planar when MIXED, else the same as OpD).
template <class OpD, class OpF, bool MIXED>
int run_cgne(const Geom& g, const OpD& opd, const OpF& opf, const SolveArgs& a) {
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

  DevMem mb64, mr64, mt64, mp64, mr32, mp32, mt32, mx32, mS, mpart, mtick, mmass;
  bool ok = mb64.alloc(sizeof(double2) * n * nsys, st) && mr64.alloc(sizeof(double2) * n * nsys, st) &&
            mt64.alloc(sizeof(double2) * n * nsys, st) && mS.alloc(sizeof(SysState) * nsys, st) &&
            mpart.alloc(sizeof(double) * pstride * nsys, st) && mtick.alloc(sizeof(unsigned) * nsys, st) &&
            mmass.alloc(sizeof(double) * nsys, st);
  if (MIXED)
    ok = ok && mr32.alloc(sizeof(float2) * n * nsys, st) && mp32.alloc(sizeof(float2) * n * nsys, st) &&
         mt32.alloc(sizeof(float2) * n * nsys, st) && mx32.alloc(sizeof(float2) * n * nsys, st);
  else
    ok = ok && mp64.alloc(sizeof(double2) * n * nsys, st);
  if (!ok) return SW_ERR_OOM;

  double2* b64 = mb64.as<double2>();
  double2* r64 = mr64.as<double2>();
  double2* t64 = mt64.as<double2>();
  SysState* S = mS.as<SysState>();
  RedBuf rb{mpart.as<double>(), mtick.as<unsigned>(), pstride};
  double* mass_d = mmass.as<double>();

  SysState* hs = nullptr;
  if (int e = pinned_states(nsys, &hs)) return e;
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

  VF fr, fp, ft, fx;
  if constexpr (MIXED) {
    fr = VF{mr32.as<float2>(), V};
    fp = VF{mp32.as<float2>(), V};
    ft = VF{mt32.as<float2>(), V};
    fx = VF{mx32.as<float2>(), V};
    cudaMemsetAsync(mp32.p, 0, sizeof(float2) * n * nsys, st);
    cudaMemsetAsync(mx32.p, 0, sizeof(float2) * n * nsys, st);
  } else {
    fr = vr;
    fp = VF{mp64.as<double2>()};
    ft = vt;
    fx = vx;
    cudaMemsetAsync(mp64.p, 0, sizeof(double2) * n * nsys, st);
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
  };
  auto iterate = [&]() {
    cg_k1<TF, OpF><<<dim3(g1, nsys), kTile, 0, st>>>(g, opf, fp, ft, bp, S, rb);
    cg_k2<TF, OpF, VF><<<dim3(g2, nsys), kTile, 0, st>>>(g, opf, ft, fp, fr, fx, bp, n, S, rb);
    cg_k3<TF, VF, NC><<<dim3(gV, nsys), 256, 0, st>>>(V, fr, fp, n, S, ST_RUNNING);
  };

  // initial residual r = b - A x0 (all systems start in NEED_RU)
  reliable_update();
  const long long max_rounds = 4LL * (a.max_iter / kChunk + 2) + 1000;
  int rc = SW_OK;
  for (long long round = 0;; ++round) {
    cudaMemcpyAsync(hs, S, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return SW_ERR_CUDA;
    bool need_ru = false, active = false;
    for (int i = 0; i < nsys; ++i) {
      const int s = hs[i].status;
      need_ru |= (s == ST_NEED_RU);
      active |= (s == ST_RUNNING || s == ST_NEED_RU || s == ST_JUST_UPDATED);
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
    for (int i = 0; i < kChunk; ++i) iterate();
    if (cudaPeekAtLastError() != cudaSuccess) return SW_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) return SW_ERR_CUDA;

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

}  // namespace swc
