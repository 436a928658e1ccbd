// Host driver of the batched CGNE solve (Eq. 2), shared by both operators.
//
// Precision modes
//   F64    x, r, p, t in FP64 (canonical layout); the residual is replaced by
//          the recomputed b - A x whenever the iterated one meets the
//          tolerance, so convergence is always decided on a true residual.
//   MIXED  inner iterations in FP32 (or on FP16 storage) on packed copies of
//          links and vectors, with reliable updates (Sleijpen & van der Vorst
//          1996): when the iterated residual falls below delta times its
//          maximum since the last update (or meets the tolerance), the FP32
//          correction is added to the FP64 solution and r = b - A x is
//          recomputed in FP64 as (D+m)^+ (chi - (D+m) x).  Dot products
//          always accumulate in FP64.
//
// The host launches iterations in chunks and reads the per-system status
// words between chunks; iterations of systems that have stopped return at
// once on the device.
#pragma once
#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "misc_kernels.cuh"
#include "ritz.h"

namespace swc {

// Tunables (sw_set_param): iterations launched between status reads, and
// the reliable-update trigger delta (update when |r| < delta max|r|) for FP32
// or FP16 stencil storage.
int param_chunk();
double param_delta(bool half);
int param_ns(int nc);  // systems per thread of the FP32 stencils (1, 2 or 4) for NC components
bool param_group_fast();     // system groups as the fastest grid dimension of the stencils
bool param_graphs();   // replay chunks of iterations as captured CUDA graphs
bool param_persistent();  // whole solve as one CUDA graph with a device-driven loop of rounds
int param_wilson_lean();  // -1 by lattice size, 0 the default form, 1 the lean form (FP32 Wilson, r = 1)

// Operators applied in two passes (the even-odd Schur complement): before
// every application the engine launches the operator's pre-pass, which
// writes the intermediate field into scratch that follows each system's
// vector; their FP64 vectors therefore take twice the per-system stride.
template <class Op, class = void> struct two_pass : std::false_type {};
template <class Op> struct two_pass<Op, std::void_t<decltype(Op::kTwoPass)>> : std::bool_constant<Op::kTwoPass> {};
template <class Op> constexpr int f64_stride_factor() { return two_pass<Op>::value ? 2 : 1; }

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
    cudaMemPool_t pool = lib_pool();
    if (!pool) return false;
    return cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, st) == cudaSuccess;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// FP16 links keep two rows and rebuild the third, which needs SU(3) links:
// SW_ERR_ARG if any link of U deviates from SU(3) by more than 1e-5.
// The lean FP32 Wilson stencil (WOp's LEAN form) for lattices whose packed
// FP32 links (288 B per site) take at most 64 MB, half the L2 -- measured on
// GB300: 3% faster at 16^3x32, 4-8% slower at 24^3x48 and 32^3x64.
inline bool wilson_lean(const Geom& g) {
  const int f = param_wilson_lean();
  return f < 0 ? (size_t)g.V * 288 <= (size_t(64) << 20) : f == 1;
}

inline int check_su3(const Geom& g, const double2* U, cudaStream_t st) {
  DevMem m;
  if (!m.alloc(sizeof(unsigned), st)) return SW_ERR_OOM;
  cudaMemsetAsync(m.p, 0, sizeof(unsigned), st);
  su3_deviation<<<sm_count() * 4, 256, 0, st>>>(g.V, U, m.as<unsigned>());
  note_launches(1);
  unsigned bits = 0;
  if (cudaMemcpyAsync(&bits, m.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SW_ERR_CUDA;
  float dev;
  std::memcpy(&dev, &bits, sizeof(dev));
  return (dev <= 1e-5f) ? SW_OK : SW_ERR_ARG;
}

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

// Pinned, mapped host buffer for the CG coefficient histories of one solve
// (per host thread, grown as needed; nullptr above 256 MB: such batches read
// them into ordinary host memory).
inline double* pinned_hist(size_t n) {
  thread_local double* buf = nullptr;
  thread_local size_t cap = 0;
  if (n * sizeof(double) > (256u << 20)) return nullptr;
  if (n > cap) {
    if (buf) cudaFreeHost(buf);
    buf = nullptr;
    cap = 0;
    if (cudaMallocHost((void**)&buf, sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cap = n;
  }
  return buf;
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
  double2 *b64, *r64, *t64;  // FP64 canonical (b64: FP64 mode only)
  void *p_lo, *t_lo;         // stencil vectors p, t in the inner precision's storage
  float2 *r32, *x32;         // FP32 residual and correction (mixed precision only)
  SysState* S;
  double* partials;
  unsigned* tickets;  // [2 nsys]: iteration kernels, then reliable-update kernels
  double* mass;
  double* hist;  // CG coefficients, [nsys][kHist][2]
  int* pcount;   // systems computed per sampled launch: [kProfSlots/2][3] (k1, k2, k3), then the FP64 samples
  int* ctl;      // device-driven solve: [0] rounds run, [1] round cap reached
};

constexpr int kProfSlots = 1024;  // sampled iterations per solve

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Bytes of workspace for nsys systems of NC complex components per site; pt:
// bytes of one system's p (or t) in the inner precision's storage.
// pt: bytes of one system's p (or t); nsys_pt: systems p and t are allocated
// for (the whole pairs of a paired layout)
inline size_t workspace_bytes_pt(int V, int NC, int nsys, bool mixed, size_t pt, int f64_factor = 1,
                                 int nsys_pt = -1) {
  if (nsys_pt < 0) nsys_pt = nsys;
  const size_t n = (size_t)V * NC * nsys * f64_factor;
  const size_t ntiles = (size_t)(V + kTile - 1) / kTile;
  size_t b = (mixed ? 2 : 3) * align_up(sizeof(double2) * n);  // b64 only in FP64 mode
  const size_t n32 = (size_t)V * NC * nsys;  // FP32 r and x carry no scratch
  b += mixed ? 2 * align_up(pt * nsys_pt) + 2 * align_up(sizeof(float2) * n32) : align_up(pt * nsys_pt);
  b += align_up(sizeof(SysState) * nsys) + align_up(sizeof(double) * 2 * kWarps * ntiles * nsys) +
       align_up(sizeof(unsigned) * 2 * nsys) + align_up(sizeof(double) * nsys) +
       align_up(sizeof(double) * 2 * kHist * nsys) + align_up(sizeof(int) * 2 * kProfSlots) +
       align_up(sizeof(int) * 8);
  return b;
}
// FP64 or FP32 storage of p and t
inline size_t workspace_bytes(int V, int NC, int nsys, bool mixed) {
  return workspace_bytes_pt(V, NC, nsys, mixed, (size_t)V * NC * (mixed ? sizeof(float2) : sizeof(double2)));
}
// f64_factor: 2 for two-pass operators, whose FP64 vectors and stencil
// vectors p, t carry their scratch after each system's field
template <class PVec> inline int pt_systems(int nsys) { return is_paired<PVec>::value ? (nsys + 1) & ~1 : nsys; }
template <class PVec> inline size_t workspace_bytes_for(int V, int NC, int nsys, bool mixed, int f64_factor = 1) {
  return workspace_bytes_pt(V, NC, nsys, mixed, sizeof(typename PVec::unit) * PVec::sys_units(V) * f64_factor,
                            f64_factor, pt_systems<PVec>(nsys));
}

inline Workspace carve_workspace_pt(void* base, int V, int NC, int nsys, bool mixed, size_t pt, int f64_factor = 1,
                                    int nsys_pt = -1) {
  if (nsys_pt < 0) nsys_pt = nsys;
  const size_t n = (size_t)V * NC * nsys * f64_factor;
  const size_t n32 = (size_t)V * NC * nsys;
  const size_t ntiles = (size_t)(V + kTile - 1) / kTile;
  char* c = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    void* p = c;
    c += align_up(bytes);
    return p;
  };
  Workspace w{};
  w.b64 = mixed ? nullptr : (double2*)take(sizeof(double2) * n);
  w.r64 = (double2*)take(sizeof(double2) * n);
  w.t64 = (double2*)take(sizeof(double2) * n);
  if (mixed) {
    w.p_lo = take(pt * nsys_pt);
    w.t_lo = take(pt * nsys_pt);
    w.r32 = (float2*)take(sizeof(float2) * n32);
    w.x32 = (float2*)take(sizeof(float2) * n32);
  } else {
    w.p_lo = take(pt * nsys_pt);
    w.t_lo = w.t64;
  }
  w.S = (SysState*)take(sizeof(SysState) * nsys);
  w.partials = (double*)take(sizeof(double) * 2 * kWarps * ntiles * nsys);  // 2nd half: norm_b's |x0|^2
  w.tickets = (unsigned*)take(sizeof(unsigned) * 2 * nsys);  // 2nd half: the reliable-update kernels
  w.mass = (double*)take(sizeof(double) * nsys);
  w.hist = (double*)take(sizeof(double) * 2 * kHist * nsys);
  w.pcount = (int*)take(sizeof(int) * 2 * kProfSlots);
  w.ctl = (int*)take(sizeof(int) * 8);
  return w;
}
inline Workspace carve_workspace(void* base, int V, int NC, int nsys, bool mixed) {
  return carve_workspace_pt(base, V, NC, nsys, mixed,
                            (size_t)V * NC * (mixed ? sizeof(float2) : sizeof(double2)));
}
template <class PVec>
inline Workspace carve_workspace_for(void* base, int V, int NC, int nsys, bool mixed, int f64_factor = 1) {
  return carve_workspace_pt(base, V, NC, nsys, mixed, sizeof(typename PVec::unit) * PVec::sys_units(V) * f64_factor,
                            f64_factor, pt_systems<PVec>(nsys));
}

// A CGNE engine: `cap` system slots on one gauge field, advanced together.
//
// Each slot carries its own scalars, mass and status word (SysState) and the
// kernels compute only the slots in the state they act on, so systems can be
// admitted, iterate, take reliable updates and finish independently.  One
// round = (admission of staged slots) + (reliable updates the last status read
// asked for) + a chunk of CG iterations + an asynchronous copy of the status
// words.  The host never waits inside a round; complete() reads the copy.
//
// Admission runs on the device: p (and the FP32 correction) cleared,
// b = (D+m)^+ chi, |b|^2 and |x0|^2, then b = 0 -> x = 0 (converged),
// x0 = 0 -> r = b exactly, otherwise an FP64 residual b - A x0.  In the mixed
// modes b is formed by the inner-precision operator (it only starts the
// iteration and scales the tolerance); every residual that decides
// convergence is r = (D+m)^+ (chi - (D+m) x) in FP64, from chi itself.
//
// OpD: FP64 operator on canonical storage.  OpF: the inner-iteration operator
// (FP32 planar when MIXED, else the same as OpD).
template <class OpD, class OpF, bool MIXED>
class Engine {
 public:
  static constexpr int NC = OpD::NC;
  using V64 = typename OpD::Vec;
  using VF = typename OpF::Vec;  // stencil vectors p, t
  using TF = typename std::conditional<MIXED, float, double>::type;
  // r and x of the inner iteration
  using VR = typename std::conditional<MIXED, typename RVecOf<VF, NC>::type, V64>::type;
  // geometry of the inner iteration: blocked site order for the packed
  // FP32/FP16 storage, the canonical order for FP64
  using GK = typename std::conditional<MIXED, GeomBlk, Geom>::type;

  // chi, x: cap slots in the canonical layout (x: initial guess in, solution
  // out).  hs_read / hs_stage: host arrays [cap] (pinned for overlap).
  // ev: event marking the status copy (nullptr: complete() syncs the stream).
  // use_graphs: replay chunks as a captured CUDA graph, run reliable updates on
  // a side stream and time launches with events when profiling is enabled;
  // all of these create driver resources, so allocation-free callers pass
  // false (they get one stream, direct launches and no timing samples).
  Engine(const Geom& g, const OpD& opd, const OpF& opf, double r, int cap, double2* chi, double2* x,
         const Workspace& ws, SysState* hs_read, SysState* hs_stage, cudaStream_t st, cudaEvent_t ev,
         bool use_graphs = true)
      : g_(g), opd_(opd), opf_(opf), r_(r), cap_(cap), chi_(chi), x_(x), ws_(ws), hr_(hs_read), hst_(hs_stage),
        st_(st), ist_(st), ev_(ev), n_((size_t)g.V * NC), s64_(n_ * f64_stride_factor<OpD>()),
        use_graphs_(use_graphs && param_graphs()),
        driver_resources_(use_graphs) {
    ntiles_ = (g.V + kTile - 1) / kTile;
    pstride_ = kWarps * ntiles_;
    gb_ = make_blocked(g, g.shape);
    if constexpr (MIXED) gk_ = gb_;
    else gk_ = g;
    gfast_ = param_group_fast() ? 1 : 0;
    rb_ = RedBuf{ws.partials, ws.tickets, pstride_, ws.hist};
    // the reliable-update kernels may run while iterations of other systems
    // run on the side: their own block tickets (per system, not per group)
    rbu_ = RedBuf{ws.partials, ws.tickets + cap, pstride_, ws.hist};
    vunits_ = VF::sys_units(g.V) * f64_stride_factor<OpF>();  // (with a two-pass operator's scratch)
    // FP64 mode: r and x are the FP64 vectors themselves (stride s64_)
    runits_ = MIXED ? VR::sys_units(g.V) : s64_;
    bp_ = BatchParams{r, runits_, s64_, vunits_};
    ns_ = MIXED ? param_ns(NC) : 1;
    ngrp_ = (cap + ns_ - 1) / ns_;
    set_grids(ngrp_);
    if constexpr (MIXED) {
      fr_ = VR{reinterpret_cast<typename VR::unit*>(ws.r32), g.V};
      fx_ = VR{reinterpret_cast<typename VR::unit*>(ws.x32), g.V};
      fp_ = VF{static_cast<typename VF::unit*>(ws.p_lo), g.V};
      ft_ = VF{static_cast<typename VF::unit*>(ws.t_lo), g.V};
    } else {
      fr_ = VR{ws.r64};
      fx_ = VR{x};
      fp_ = VF{static_cast<double2*>(ws.p_lo)};
      ft_ = VF{ws.t64};
    }
    reported_.assign(cap, 1);
    for (int i = 0; i < cap; ++i) {
      SysState z{};
      z.status = ST_IDLE;
      hr_[i] = z;
    }
    cudaMemsetAsync(ws.tickets, 0, sizeof(unsigned) * 2 * cap, st);
    if (driver_resources_) {  // callers that allow driver resources get the overlapped reliable update
      if (cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        side_ = nullptr;
      }
    }
    cudaMemsetAsync(ws.pcount, 0, sizeof(int) * 2 * kProfSlots, st);
    hrd_ = mapped_alias(hr_);
    hstd_ = mapped_alias(hst_);
    move_states(ws.S, hr_, hrd_, cap, cudaMemcpyHostToDevice);
    chunk_ = param_chunk();
    delta_ = param_delta(std::is_same<VF, VecP16<NC>>::value);
  }

  // FP64 matvec launches (right-hand side: 1 application; residual: 2) are
  // timed with events and count the systems they compute.
  struct FpSample {
    cudaEvent_t e0, e1;
    int* cnt;
    int apps;
  };
  FpSample* fp_sample(int apps, cudaStream_t sx) {
    if (!prof() || fsamples_.size() >= (size_t)kProfSlots / 2) return nullptr;
    FpSample f{prof_event(), prof_event(), ws_.pcount + 2 * kProfSlots - 1 - fsamples_.size(), apps};
    cudaEventRecord(f.e0, sx);
    fsamples_.push_back(f);
    return &fsamples_.back();
  }

  // Profiler class names: "<operator>.<kernel>.<precision>".
  static const char* cls_k1() {
    static const std::string c = std::string(OpF::kName) + ".k1." + OpF::kPrec;
    return c.c_str();
  }
  static const char* cls_k2() {
    static const std::string c = std::string(OpF::kName) + ".k2." + OpF::kPrec;
    return c.c_str();
  }
  static const char* cls_k3() {
    static const std::string c = std::string(OpF::kName) + ".k3." + OpF::kPrec;
    return c.c_str();
  }
  static const char* cls_ru() {
    static const std::string c = std::string(OpD::kName) + ".ru.f64";
    return c.c_str();
  }
  static const char* cls_rhs() {
    static const std::string c = std::string(OpD::kName) + ".rhs.f64";
    return c.c_str();
  }

  // Turn the sampled launches into profiler records (after the stream is idle).
  void flush_profile() {
    flush_fp_samples();
    if (samples_.empty()) return;
    std::vector<int> cnt(3 * samples_.size());
    if (cnt.empty() ||
        cudaMemcpy(cnt.data(), ws_.pcount, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    // bytes of the stored gauge data (links, transports) and of one system's
    // stencil vector (p or t) and inner-precision vector (r or x)
    const double gauge = (double)g_.V * OpF::kGaugeBytes;
    const double pv = (double)sizeof(typename VF::unit) * VF::sys_units(g_.V);
    const double rv = (double)sizeof(typename VR::unit) * VR::sys_units(g_.V);
    // flops: the paper's count per site and application (Eq. 4) for every
    // computed system (k2's r update is not counted)
    const double fl = OpF::kFlops * g_.V;
    // k3: r, p, x read, p and x written (a streaming kernel: no flops counted)
    for (size_t k = 0; k < samples_.size(); ++k) {
      prof_push(cls_k1(), samples_[k].e0, samples_[k].e1, gauge + cnt[3 * k] * 2.0 * pv, fl * cnt[3 * k]);
      prof_push(cls_k2(), samples_[k].e1, samples_[k].e2, gauge + cnt[3 * k + 1] * (pv + 2.0 * rv),
                fl * cnt[3 * k + 1]);
      prof_push(cls_k3(), samples_[k].e2, samples_[k].e3, cnt[3 * k + 2] * (2.0 * pv + 3.0 * rv));
    }
    prof_commit(true);
    samples_.clear();
    cudaMemset(ws_.pcount, 0, sizeof(int) * 3 * kProfSlots / 2);
  }

  ~Engine() {
    for (auto& ge : gexecs_) cudaGraphExecDestroy(ge.second);
    if (side_) {
      cudaStreamSynchronize(side_);
      cudaStreamDestroy(side_);
    }
    if (ev_fork_) cudaEventDestroy(ev_fork_);
    if (ev_join_) cudaEventDestroy(ev_join_);
  }
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  int cap() const { return cap_; }
  size_t slot_elems() const { return n_; }
  double2* chi_slot(int i) const { return chi_ + (size_t)i * s64_; }
  double2* x_slot(int i) const { return x_ + (size_t)i * s64_; }
  const SysState& state(int i) const { return hr_[i]; }
  const double* hist() const { return ws_.hist; }
  cudaStream_t stream() const { return st_; }

  // Host: put slot i up for admission in the next round.  Its chi and initial
  // guess must be in the slot's buffers (in stream order) before issue().
  // cb2: |b|^2 of the convergence criterion of an operator that has its own
  // (full_conv; 0: the iterated system's).
  void stage(int i, double mass, double tol, int max_iter, double cb2 = 0.0) {
    SysState s{};
    s.tol2 = tol * tol;
    s.cb2 = cb2;
    s.delta2 = MIXED ? delta_ * delta_ : 0.0;
    s.max_iter = max_iter;
    s.mass = mass;
    s.status = ST_ADMIT;
    hst_[i] = s;
    hr_[i].status = ST_ADMIT;
    reported_[i] = 0;
    staged_.push_back(i);
  }

  // Launch one round on the stream (see the class comment).
  void issue() {
    SysState* S = ws_.S;
    bool ru = need_ru_;
    // Grids of the launches that compute only some slots (admission, reliable
    // updates) are sized for the slots they compute, not for the engine's
    // capacity: the blocks of the other slots return at once, and a launch
    // sized for all slots would leave the SMs nearly empty (the FP64
    // matvecs need full occupancy to keep the FP64 pipe busy).
    int n_ru = need_ru_ ? nneed_ : 0;
    if (!staged_.empty()) {
      const int na = (int)staged_.size();
      n_ru += na;  // admitted systems with a guess x0 != 0 take an FP64 residual now
      upload_staged();
      admit(na);
      ru = true;
    }
    // After reliable updates with nothing known to be running, read the
    // statuses first rather than launch a chunk that may find nothing to do.
    const bool run = !ru || nrun_ > 0;
    // The reliable update (FP64, bound by the FP64 pipe) runs on the side
    // stream while the chunk of iterations of the other systems (FP32, bound
    // by memory) runs on the engine's stream: they act on disjoint systems.
    const bool overlap = ru && run && side_ != nullptr;
    if (ru) {
      mark_ru<<<(cap_ + 127) / 128, 128, 0, st_>>>(cap_, S);
      launches(1);
      if (overlap) {
        cudaEventRecord(ev_fork_, st_);
        cudaStreamWaitEvent(side_, ev_fork_, 0);
        reliable_update(n_ru, side_);
        cudaEventRecord(ev_join_, side_);
      } else {
        reliable_update(n_ru, st_);
      }
    }
    if (run) {
      size_for_live();
      // every 4th chunk is timed when profiling, on its second iteration: by
      // then the queue is full, so the events time the kernels rather than the
      // host's launch latency
      // (never in a round whose reliable update runs alongside: the events
      // would time the two streams' kernels sharing the GPU)
      const bool prof = this->prof() && chunk_ > 1 && samples_.size() < (size_t)kProfSlots / 2 &&
                        (chunks_ % 4 == 0) && !overlap;
      ++chunks_;
      if (!prof && use_graphs_ && chunks_ > 1) {
        launch_chunk_graph();
      } else {
        for (int i = 0; i < chunk_; ++i) iterate(prof && i == 1);
      }
    }
    if (overlap) cudaStreamWaitEvent(st_, ev_join_, 0);
    move_states(hr_, S, hrd_, cap_, cudaMemcpyDeviceToHost);
    if (ev_) cudaEventRecord(ev_, st_);
  }

  // The round's status copy has landed (non-blocking check).
  bool ready() const { return ev_ ? cudaEventQuery(ev_) != cudaErrorNotReady : true; }

  // Wait for the round and scan the status words.  Returns the number of
  // slots still in flight, or a negative SW_ERR_* code.
  int complete() {
    const cudaError_t e = ev_ ? cudaEventSynchronize(ev_) : cudaStreamSynchronize(st_);
    if (e != cudaSuccess) return cuda_fail(e);
    if (const cudaError_t l = cudaGetLastError(); l != cudaSuccess) return cuda_fail(l);
    const int active = complete_scan();
    ++rounds_;
    return active;
  }

  // Scan the status words read back (the host copy hr_).
  int complete_scan() {
    int active = 0, nrun = 0;
    need_ru_ = false;
    nneed_ = 0;
    for (int i = 0; i < cap_; ++i) {
      const int s = hr_[i].status;
      need_ru_ |= (s == ST_NEED_RU);
      nneed_ += (s == ST_NEED_RU);
      nrun += (s == ST_RUNNING);
      active += (s == ST_RUNNING || s == ST_NEED_RU || s == ST_JUST_UPDATED || s == ST_ADMIT ||
                 s == ST_ZERO_B || s == ST_ZERO_GUESS || s == ST_RU_PENDING || s == ST_READY);
    }
    nrun_ = nrun;
    return active;
  }

  // Slots that reached a final state since the last call (each reported once).
  void finished(std::vector<int>& out) {
    for (int i = 0; i < cap_; ++i) {
      const int s = hr_[i].status;
      if (!reported_[i] && (s == ST_CONVERGED || s == ST_MAXITER || s == ST_FAILED)) {
        reported_[i] = 1;
        out.push_back(i);
      }
    }
  }

  // Whether this engine may run a solve as one device-driven CUDA graph
  // (it needs driver resources, and the kernel-timing samples need the
  // host-driven rounds).
  bool can_persist() const { return driver_resources_ && side_ != nullptr && !prof(); }

  // Solve the staged systems with one launch of one CUDA graph: the
  // admission kernels, then a conditional WHILE node whose body is one round
  // -- the start of the reliable updates the statuses ask for (NEED_RU ->
  // RU_PENDING), their FP64 kernels on a parallel branch beside a chunk of
  // iterations of the running systems, then round_end, which keeps the loop
  // going while any system is in flight (at most max_rounds rounds, else a
  // timeout) -- and the copy of the status words to the host.  The host
  // launches once and waits once.  The rounds are those of the host-driven
  // loop, and a system's arithmetic does not depend on when its update runs
  // beside the other systems' iterations, so the results are the same bit for
  // bit.  Grids are sized for every slot: as systems finish, their blocks
  // return at once.  Returns the number of slots still in flight (0), or a
  // negative SW_ERR_* code; SW_ERR_CUDA before anything was launched means the
  // graph could not be built (the caller then runs host-driven rounds).
  int solve_persistent(int max_rounds, bool* launched) {
    *launched = false;
    if (staged_.empty()) return 0;
    const int na = (int)staged_.size();
    upload_staged();
    set_grids(ngrp_);
    SysState* S = ws_.S;
    cudaMemsetAsync(ws_.ctl, 0, sizeof(int) * 8, st_);
    cudaStream_t body_st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamCreateWithFlags(&body_st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int per_round = 0;
    if (ok) {
      capturing_ = true;
      admit(na);
      cudaStreamCaptureStatus cs;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      cudaGraphConditionalHandle loop = 0;
      cudaGraphNode_t wnode = nullptr;
      cudaGraphNodeParams cp{};
      ok = cudaStreamGetCaptureInfo(st_, &cs, nullptr, &cg, &deps, nullptr, &ndeps) == cudaSuccess &&
           cs == cudaStreamCaptureStatusActive &&
           cudaGraphConditionalHandleCreate(&loop, cg, 1, cudaGraphCondAssignDefault) == cudaSuccess;
      if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp) == cudaSuccess;
      }
      if (ok) {  // the loop body: one round
        ok = cudaStreamBeginCaptureToGraph(body_st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          ist_ = body_st;
          mark_ru<<<(cap_ + 127) / 128, 128, 0, body_st>>>(cap_, S);
          cudaEventRecord(ev_fork_, body_st);
          cudaStreamWaitEvent(side_, ev_fork_, 0);
          reliable_update(cap_, side_);
          cudaEventRecord(ev_join_, side_);
          for (int i = 0; i < chunk_; ++i) iterate(false, false);
          cudaStreamWaitEvent(body_st, ev_join_, 0);
          round_end<<<1, 256, 0, body_st>>>(cap_, S, ws_.ctl, max_rounds, loop);
          ist_ = st_;
          cudaGraph_t body = nullptr;
          ok = cudaStreamEndCapture(body_st, &body) == cudaSuccess;
          per_round = 2 + (MIXED ? 7 : 5) + 4 * chunk_ + (two_pass<OpF>::value ? 2 * chunk_ + 2 : 0);
        }
      }
      ok = ok && cudaStreamUpdateCaptureDependencies(st_, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                     cudaSuccess;
      move_states(hr_, S, hrd_, cap_, cudaMemcpyDeviceToHost);
      cudaGraph_t done = nullptr;
      ok = (cudaStreamEndCapture(st_, &done) == cudaSuccess) && ok && done;
      graph = done;
      ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    }
    capturing_ = false;
    if (graph) cudaGraphDestroy(graph);
    if (body_st) cudaStreamDestroy(body_st);
    ist_ = st_;
    if (!ok) {
      if (exec) cudaGraphExecDestroy(exec);
      cudaGetLastError();
      // nothing of the solve ran: restage for the host-driven rounds
      for (int i = 0; i < cap_; ++i)
        if (hr_[i].status == ST_ADMIT) staged_.push_back(i);
      return SW_ERR_CUDA;
    }
    const cudaError_t le = cudaGraphLaunch(exec, st_);
    *launched = le == cudaSuccess;
    const cudaError_t se = cudaStreamSynchronize(st_);
    cudaGraphExecDestroy(exec);
    if (le != cudaSuccess) return cuda_fail(le);
    if (se != cudaSuccess) return cuda_fail(se);
    int ctl[2] = {0, 0};
    if (const cudaError_t e = cudaMemcpy(ctl, ws_.ctl, sizeof(ctl), cudaMemcpyDeviceToHost); e != cudaSuccess)
      return cuda_fail(e);
    note_launches(6 + ctl[0] * per_round + 1);
    rounds_ += ctl[0];
    if (ctl[1]) return SW_ERR_TIMEOUT;
    const int active = complete_scan();
    return active;
  }

  long long rounds() const { return rounds_; }

 private:
  // The pre-pass of a two-pass operator (nothing for the others): the
  // intermediate field of `in`'s systems in `status`, before the operator
  // is applied to them.
  template <class Op, class Vec>
  void prepass(const Op& op, const Vec& in, size_t stride, int status, bool dagger, cudaStream_t s) {
    if constexpr (two_pass<Op>::value) {
      op.prepass(in, stride, ws_.S, status, dagger ? 1 : 0, cap_, s);
      launches(1);
    }
  }

  // Admission launches for the na slots staged (their status words already on
  // the device): see the class comment.
  void admit(int na) {
    SysState* S = ws_.S;
    const int gv = grid_of((const void*)admit_clear<VF, NC>, 256, na);
    admit_clear<VF, NC><<<dim3(gv, cap_), 256, 0, st_>>>(g_.V, fp_, vunits_, MIXED ? ws_.x32 : nullptr,
                                                         MIXED ? n_ : 0, S);
    const int gn = grid_of((const void*)norm_b<NC>, kTile, na);
    if constexpr (MIXED) {
      // b = (D+m)^+ chi in the inner precision: r = p = b and |b|^2
      demote_chi<NC, VF><<<dim3(grid_of((const void*)demote_chi<NC, VF>, 256, na), cap_), 256, 0, st_>>>(
          gb_, chi_, ft_, s64_, vunits_, S);
      prepass(opf_, ft_, vunits_, ST_ADMIT, true, st_);
      rhs_lo<TF, OpF, VR, GK><<<dim3(grid_of((const void*)rhs_lo<TF, OpF, VR, GK>, kTile, na), cap_), kTile, 0,
                                st_>>>(gk_, opf_, ft_, fp_, fr_, bp_, S, rb_);
      norm_b<NC><<<dim3(gn, cap_), kTile, 0, st_>>>(g_.V, nullptr, x_, s64_, S, rb_);
      admit_vectors<NC><<<dim3(gv, cap_), 256, 0, st_>>>(g_.V, x_, ws_.r64, nullptr, s64_, S);
      launches(1);
    } else {
      FpSample* fs = fp_sample(1, st_);
      if (prof()) prof_count(cls_rhs(), 1);
      prepass(opd_, V64{chi_}, s64_, ST_ADMIT, true, st_);
      apply_kernel<double, OpD><<<dim3(grid_of((const void*)apply_kernel<double, OpD>, kTile, na), cap_), kTile,
                                  0, st_>>>(g_, opd_, V64{chi_}, V64{ws_.b64}, 0.0, s64_, r_, 1, S, ST_ADMIT,
                                            fs ? fs->cnt : nullptr);
      if (fs) cudaEventRecord(fs->e1, st_);
      norm_b<NC><<<dim3(gn, cap_), kTile, 0, st_>>>(g_.V, ws_.b64, x_, s64_, S, rb_);
      admit_vectors<NC><<<dim3(gv, cap_), 256, 0, st_>>>(g_.V, x_, ws_.r64, ws_.b64, s64_, S);
    }
    admit_states<<<(cap_ + 127) / 128, 128, 0, st_>>>(cap_, S, MIXED ? 1 : 0);
    launches(5);
  }

  // Device address of a host status buffer that is pinned and mapped, else
  // nullptr (ordinary host memory, e.g. the allocation-free entry's).
  static SysState* mapped_alias(SysState* h) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer ? static_cast<SysState*>(at.devicePointer) : nullptr;
  }

  // n status words between the device and the host buffer `h` (device alias
  // `hd`), in stream order on the engine's stream: by kernel when the host
  // buffer is mapped, so the transfer does not wait behind copies the caller
  // has queued on the copy engines, else by cudaMemcpyAsync.
  void move_states(SysState* dst, const SysState* src, SysState* hd, int n, cudaMemcpyKind kind) {
    if (n <= 0) return;
    if (hd) {
      const size_t words = sizeof(SysState) / 8 * (size_t)n;
      const SysState* from = kind == cudaMemcpyHostToDevice ? hd : src;
      SysState* to = kind == cudaMemcpyHostToDevice ? dst : hd;
      const int blocks = (int)std::min<size_t>((words + 255) / 256, (size_t)sm_count());
      copy_words<<<blocks, 256, 0, st_>>>(reinterpret_cast<const unsigned long long*>(from),
                                          reinterpret_cast<unsigned long long*>(to), words);
      launches(1);
    } else {
      cudaMemcpyAsync(dst, src, sizeof(SysState) * n, kind, st_);
    }
  }

  void upload_staged() {
    std::sort(staged_.begin(), staged_.end());
    size_t a = 0;
    while (a < staged_.size()) {  // one copy per run of consecutive slots
      size_t b = a + 1;
      while (b < staged_.size() && staged_[b] == staged_[b - 1] + 1) ++b;
      move_states(ws_.S + staged_[a], hst_ + staged_[a], hstd_ ? hstd_ + staged_[a] : nullptr, (int)(b - a),
                  cudaMemcpyHostToDevice);
      a = b;
    }
    staged_.clear();
  }

  // The reliable update of the systems in RU_PENDING, on stream `sx`.
  // nsys: the slots (at most) that take the update this round, for the grids.
  void reliable_update(int nsys, cudaStream_t sx) {
    SysState* S = ws_.S;
    const int gv = grid_of((const void*)cg_k3<TF, VR, VF, NC>, 256, nsys);
    const int g3 = grid_of(k3_ptr(), 256, k3_rows(nsys));
    // the last x += alpha p of each system (k2 stopped it before k3)
    launch_k3(g3, ST_RU_PENDING, 1, sx, nullptr);
    if constexpr (MIXED) accum_x<NC, VR><<<dim3(gv, cap_), 256, 0, sx>>>(gb_, x_, fx_, s64_, runits_, S);
    FpSample* fs = fp_sample(2, sx);
    if (prof()) prof_count(cls_ru(), 1);
    // r = (D+m)^+ (chi - (D+m) x) = b - A x, all in FP64
    prepass(opd_, V64{x_}, s64_, ST_RU_PENDING, false, sx);
    apply_kernel<double, OpD><<<dim3(grid_of((const void*)apply_kernel<double, OpD>, kTile, nsys), cap_), kTile, 0,
                                sx>>>(g_, opd_, V64{x_}, V64{ws_.t64}, 0.0, s64_, r_, 0, S, ST_RU_PENDING,
                                      fs ? fs->cnt : nullptr, V64{chi_}, 1);
    prepass(opd_, V64{ws_.t64}, s64_, ST_RU_PENDING, true, sx);
    residual64<OpD><<<dim3(grid_of((const void*)residual64<OpD>, kTile, nsys), cap_), kTile, 0, sx>>>(
        g_, opd_, V64{ws_.t64}, V64{ws_.r64}, bp_, S, rbu_);
    if (fs) cudaEventRecord(fs->e1, sx);
    if constexpr (MIXED) demote_r<NC, VR><<<dim3(gv, cap_), 256, 0, sx>>>(gb_, ws_.r64, fr_, s64_, runits_, S);
    launch_k3(g3, ST_JUST_UPDATED, 2, sx, nullptr);
    mark_ready<<<(cap_ + 127) / 128, 128, 0, sx>>>(cap_, S);
    launches(MIXED ? 7 : 5);
  }

  // One graph per grid class (see size_for_live), captured on first use.
  void launch_chunk_graph() {
    cudaGraphExec_t ge = nullptr;
    for (auto& g : gexecs_)
      if (g.first == cls_) ge = g.second;
    if (!ge && !graph_failed_) {
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        for (int i = 0; i < chunk_; ++i) iterate(false, false);
        ok = cudaStreamEndCapture(st_, &graph) == cudaSuccess && graph;
      }
      ok = ok && cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      if (!ok) {
        cudaGetLastError();
        ge = nullptr;
        graph_failed_ = true;
      } else {
        gexecs_.push_back({cls_, ge});
      }
    }
    if (ge) {
      cudaGraphLaunch(ge, st_);
      launches(4 * chunk_);
      if (prof()) {
        prof_count(cls_k1(), chunk_);
        prof_count(cls_k2(), chunk_);
        prof_count(cls_k3(), chunk_);
      }
    } else {
      for (int i = 0; i < chunk_; ++i) iterate(false);
    }
  }

  // Grids of the iteration kernels for `groups` groups of ns_ slots that may
  // run (blocks of stopped slots return at once).
  void set_grids(int groups) {
    cls_ = groups;
    g1_ = grid_for(k1_ptr(), kTile, g_.V, groups, ntiles_);
    g2_ = grid_for(k2_ptr(), kTile, g_.V, groups, ntiles_);
    gV_ = grid_for(k3_ptr(), 256, g_.V, k3_rows(groups * ns_), ntiles_);
  }

  // Size the iteration grids for the groups holding a slot that may run in
  // the next chunk, rounded up to a power of two (at most the engine's
  // groups): as systems converge, the remaining ones keep the SMs full.  A
  // system's arithmetic and reduction order do not depend on the grid.
  void size_for_live() {
    int live = 0;
    for (int gi = 0; gi < ngrp_; ++gi) {
      bool any = false;
      for (int i = gi * ns_; i < cap_ && i < (gi + 1) * ns_; ++i) {
        const int s = hr_[i].status;
        any |= (s == ST_RUNNING || s == ST_NEED_RU || s == ST_JUST_UPDATED || s == ST_ADMIT || s == ST_ZERO_GUESS ||
                s == ST_READY);
      }
      live += any;
    }
    int cls = 1;
    while (cls < live) cls *= 2;
    if (cls > ngrp_) cls = ngrp_;
    if (cls != cls_) set_grids(cls);
  }

  void flush_fp_samples() {
    if (fsamples_.empty()) return;
    std::vector<int> cnt(2 * kProfSlots);
    if (cudaMemcpy(cnt.data(), ws_.pcount, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    for (size_t k = 0; k < fsamples_.size(); ++k) {
      const FpSample& f = fsamples_[k];
      const int systems = cnt[2 * kProfSlots - 1 - k];
      prof_push(f.apps == 2 ? cls_ru() : cls_rhs(), f.e0, f.e1, 0.0,
                OpD::kFlops * g_.V * f.apps * systems);
    }
    prof_commit(true);
    fsamples_.clear();
    cudaMemset(ws_.pcount + 3 * kProfSlots / 2, 0, sizeof(int) * kProfSlots / 2);
  }

  // Register-blocking widths 2 and 4 exist for the inner-precision stencils
  // only (the FP64 ones are ALU-bound and run one system per thread).
  const void* k1_ptr() const {
    if constexpr (MIXED) {
      if (ns_ == 2) return (const void*)cg_k1<TF, OpF, 2, GK>;
      if (ns_ == 4) return (const void*)cg_k1<TF, OpF, 4, GK>;
    }
    return (const void*)cg_k1<TF, OpF, 1, GK>;
  }
  const void* k2_ptr() const {
    if constexpr (MIXED) {
      if (ns_ == 2) return (const void*)cg_k2<TF, OpF, 2, VR, GK>;
      if (ns_ == 4) return (const void*)cg_k2<TF, OpF, 4, VR, GK>;
    }
    return (const void*)cg_k2<TF, OpF, 1, VR, GK>;
  }
  template <int NS> void launch_k12(int* c) {
    SysState* S = ws_.S;
    const dim3 grid1 = gfast_ ? dim3(ngrp_, g1_) : dim3(g1_, ngrp_), grid2 = gfast_ ? dim3(ngrp_, g2_) : dim3(g2_, ngrp_);
    prepass(opf_, fp_, vunits_, ST_RUNNING, false, ist_);
    cg_k1<TF, OpF, NS, GK><<<grid1, kTile, 0, ist_>>>(gk_, opf_, fp_, ft_, bp_, cap_, S, rb_, c, gfast_);
    if (c) cudaEventRecord(samples_.back().e1, ist_);
    prepass(opf_, ft_, vunits_, ST_RUNNING, true, ist_);
    cg_k2<TF, OpF, NS, VR, GK><<<grid2, kTile, 0, ist_>>>(gk_, opf_, ft_, fr_, bp_, cap_, S, rb_,
                                                          c ? c + 1 : nullptr, gfast_);
  }

  // One CG iteration (k1, k2, k3).  A sampled iteration is bracketed by
  // events, and its stencil kernels count the systems they compute; the
  // algorithmic bytes of a launch (every stored element touched once) are the
  // links (and transports) once plus, per computed system, the vectors read
  // and written: k1 p read, t written; k2 t read, r read and written.
  void iterate(bool sample, bool count = true) {
    SysState* S = ws_.S;
    int* c = nullptr;
    if (sample) {
      samples_.push_back(Sample{prof_event(), prof_event(), prof_event(), prof_event()});
      c = ws_.pcount + 3 * (samples_.size() - 1);
      cudaEventRecord(samples_.back().e0, ist_);
    }
    commit_ready<<<(cap_ + 127) / 128, 128, 0, ist_>>>(cap_, S);
    if constexpr (MIXED) {
      if (ns_ == 2) launch_k12<2>(c);
      else if (ns_ == 4) launch_k12<4>(c);
      else launch_k12<1>(c);
    } else {
      launch_k12<1>(c);
    }
    if (sample) cudaEventRecord(samples_.back().e2, ist_);
    launch_k3(gV_, ST_RUNNING, 3, ist_, c ? c + 2 : nullptr);
    if (sample) cudaEventRecord(samples_.back().e3, ist_);
    if (count) {
      launches(4);
      if (prof()) {
        prof_count(cls_k1(), 1);
        prof_count(cls_k2(), 1);
        prof_count(cls_k3(), 1);
      }
    }
  }

  struct Sample {
    cudaEvent_t e0, e1, e2, e3;
  };
  Geom g_;
  GK gk_;
  GeomBlk gb_;
  OpD opd_;
  OpF opf_;
  double r_;
  int cap_;
  double2* chi_;
  double2* x_;
  Workspace ws_;
  SysState* hr_;
  SysState* hst_;
  SysState* hrd_ = nullptr;   // device alias of hr_ when mapped
  SysState* hstd_ = nullptr;  // device alias of hst_ when mapped
  cudaStream_t st_;
  cudaStream_t ist_;  // stream the iteration kernels go to (st_, or the loop body's capture stream)
  cudaEvent_t ev_;
  size_t n_;    // complex components of one system's field (g.V x NC)
  size_t s64_;  // per-system stride of the FP64 vectors (n_, or 2 n_ with a two-pass operator's scratch)
  int ntiles_ = 0, pstride_ = 0, ngrp_ = 0, gV_ = 0, g1_ = 0, g2_ = 0;
  RedBuf rb_{}, rbu_{};
  cudaStream_t side_ = nullptr;  // reliable updates overlapped with iterations
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  BatchParams bp_{};
  VF fp_{}, ft_{};
  VR fr_{}, fx_{};
  size_t vunits_ = 0, runits_ = 0;  // storage units of one system's p (t) and r (x)
  int chunk_ = 16;
  double delta_ = 0.1;
  bool need_ru_ = false;
  int nneed_ = 0;  // slots in NEED_RU at the last status read

  // Blocks per slot of a launch that computes `nsys` of the engine's slots.
  // k3 (x += alpha p and/or p = r + beta p, by `mode` bits) on the systems in
  // `status`: one row of blocks per system, or per pair of systems when p
  // is paired
  static const void* k3_ptr() {
    if constexpr (is_paired<VF>::value) return (const void*)cg_k3_pair<VR, VF, NC>;
    else return (const void*)cg_k3<TF, VR, VF, NC>;
  }
  static int k3_rows(int nsys) { return is_paired<VF>::value ? (nsys + 1) / 2 : nsys; }
  void launch_k3(int gx, int status, int mode, cudaStream_t s, int* nact) const {
    if constexpr (is_paired<VF>::value)
      cg_k3_pair<VR, VF, NC><<<dim3(gx, k3_rows(cap_)), 256, 0, s>>>(g_.V, fr_, fp_, fx_, runits_, vunits_, ws_.S,
                                                                     cap_, status, mode, nact);
    else
      cg_k3<TF, VR, VF, NC><<<dim3(gx, cap_), 256, 0, s>>>(g_.V, fr_, fp_, fx_, runits_, vunits_, ws_.S, status,
                                                           mode, nact);
  }
  int grid_of(const void* kernel, int block, int nsys) const {
    return grid_for(kernel, block, g_.V, nsys < 1 ? 1 : (nsys > cap_ ? cap_ : nsys), ntiles_);
  }
  int nrun_ = 0, ns_ = 1, gfast_ = 0;
  std::vector<Sample> samples_;
  std::vector<FpSample> fsamples_;
  long long rounds_ = 0, chunks_ = 0;
  bool use_graphs_ = true, graph_failed_ = false;
  bool driver_resources_ = true;  // false: allocation-free caller (no side stream, graphs or timing events)
  bool prof() const { return driver_resources_ && prof_enabled(); }
  bool capturing_ = false;  // building the device-driven solve's graph: its launches are counted when it runs
  void launches(int k) const {
    if (!capturing_) note_launches(k);
  }
  int cls_ = 0;  // groups the iteration grids are sized for
  std::vector<std::pair<int, cudaGraphExec_t>> gexecs_;
  std::vector<int> staged_;
  std::vector<char> reported_;
};

// Fill sw_solve_info for slot i of an engine from its final status word and
// its CG coefficients (hh: host copy of the slot's [kHist][2] history).
inline int fill_info(const SysState& s, const double* hh, int precision, double secs, sw_solve_info* inf) {
  const int code = status_to_code(s.status);
  if (inf) {
    inf->iters = s.iter;
    inf->reliable_updates = s.n_ru;
    inf->status = code;
    inf->precision = precision;
    const double b2 = s.cb2 > 0.0 ? s.cb2 : s.b2;
    inf->true_rel_resid = b2 > 0 ? sqrt(s.rr_true / b2) : 0.0;
    inf->seconds = secs;
    ritz_extremes(hh, s.iter < kHist ? s.iter : kHist, &inf->lambda_min, &inf->lambda_max);
  }
  return code;
}

inline int worst_code(int worst, int code) {
  if (code < 0 && (worst >= 0 || code < worst)) return code;
  if (code > 0 && worst == SW_OK) return code;
  return worst;
}

// Batched solve on caller-provided workspace: every system admitted at once,
// rounds until none is in flight.  hs: host array [2 nsys] (status reads and
// staging).
template <class OpD, class OpF, bool MIXED>
int run_cgne_ws(const Geom& g, const OpD& opd, const OpF& opf, const SolveArgs& a, const Workspace& ws,
                SysState* hs, bool use_graphs = true, double* hist_host = nullptr) {
  using namespace std::chrono;
  const auto t0 = steady_clock::now();
  Engine<OpD, OpF, MIXED> e(g, opd, opf, a.r, a.nsys, const_cast<double2*>(a.chi), a.x, ws, hs, hs + a.nsys,
                            a.stream, nullptr, use_graphs);
  for (int i = 0; i < a.nsys; ++i)
    e.stage(i, a.masses[i], a.tols ? a.tols[i] : a.tol, a.max_iter, a.conv_b2 ? a.conv_b2[i] : 0.0);
  const long long max_rounds = 4LL * (a.max_iter / param_chunk() + 2) + 1000;
  int rc = SW_OK;
  bool host_rounds = true;
  if (param_persistent() && e.can_persist()) {
    bool launched = false;
    const int p = e.solve_persistent((int)std::min<long long>(max_rounds, 1 << 30), &launched);
    if (p == SW_ERR_TIMEOUT) {
      rc = SW_ERR_TIMEOUT;
      host_rounds = false;
    } else if (p < 0 && launched) {
      return p;
    } else if (p >= 0) {
      host_rounds = p > 0;  // (0: every system finished on the device)
    }
  }
  for (; host_rounds;) {
    e.issue();
    const int active = e.complete();
    if (active < 0) return active;
    if (active == 0) break;
    if (e.rounds() > max_rounds) {
      rc = SW_ERR_TIMEOUT;
      break;
    }
  }
  e.flush_profile();
  prof_flush();
  // the CG coefficients, for the Ritz values: by kernel into mapped pinned
  // memory when the caller has such a buffer (so the read does not queue
  // behind bulk copies on a copy engine), else by cudaMemcpyAsync
  std::vector<double> hv;
  const double* hh = nullptr;
  if (a.infos) {
    const size_t nh = (size_t)2 * kHist * a.nsys;
    void* hist_dev = nullptr;
    if (hist_host && cudaHostGetDevicePointer(&hist_dev, hist_host, 0) != cudaSuccess) {
      cudaGetLastError();  // not mapped: read by cudaMemcpyAsync below
      hist_dev = nullptr;
    }
    if (hist_dev) {
      const int blocks = (int)std::min<size_t>((nh + 255) / 256, (size_t)sm_count() * 4);
      copy_words<<<blocks, 256, 0, a.stream>>>(reinterpret_cast<const unsigned long long*>(ws.hist),
                                               static_cast<unsigned long long*>(hist_dev), nh);
      note_launches(1);
      hh = hist_host;
    } else {
      hv.resize(nh);
      if (cudaMemcpyAsync(hv.data(), ws.hist, sizeof(double) * nh, cudaMemcpyDeviceToHost, a.stream) != cudaSuccess)
        return SW_ERR_CUDA;
      hh = hv.data();
    }
    if (cudaStreamSynchronize(a.stream) != cudaSuccess) return SW_ERR_CUDA;
  }
  const double secs = duration<double>(steady_clock::now() - t0).count();
  int worst = SW_OK;
  for (int i = 0; i < a.nsys; ++i) {
    int code = fill_info(e.state(i), a.infos ? hh + (size_t)i * 2 * kHist : nullptr, a.precision, secs,
                         a.infos ? a.infos + i : nullptr);
    if (rc != SW_OK) code = rc;
    if (a.infos && rc != SW_OK) a.infos[i].status = rc;
    worst = worst_code(worst, code);
  }
  return worst;
}

// Allocating entry: one stream-ordered block of workspace for the call and a
// pinned host buffer for the status words.
template <class OpD, class OpF, bool MIXED>
int run_cgne(const Geom& g, const OpD& opd, const OpF& opf, const SolveArgs& a) {
  using VF = typename OpF::Vec;
  DevMem mem;
  constexpr int f = f64_stride_factor<OpD>();
  if (!mem.alloc(workspace_bytes_for<VF>(g.V, OpD::NC, a.nsys, MIXED, f), a.stream)) return SW_ERR_OOM;
  SysState* hs = nullptr;
  if (int e = pinned_states(2 * a.nsys, &hs)) return e;
  const Workspace ws = carve_workspace_for<VF>(mem.p, g.V, OpD::NC, a.nsys, MIXED, f);
  return run_cgne_ws<OpD, OpF, MIXED>(g, opd, opf, a, ws, hs, true,
                                      a.infos ? pinned_hist((size_t)2 * kHist * a.nsys) : nullptr);
}


// The inner-precision operator of the mixed modes applied to nsys systems by
// the CG iteration kernels themselves: (D+m) in by cg_k1 (t = (D+m) p, with p
// the inner-precision copy of `in`), (D+m)^+ in by cg_k2 (r -= alpha (D+m)^+ t
// with r = 0, alpha = -1, t the copy of `in`), at the register-blocking width
// and site order the solves use.  in, out: canonical FP64 [nsys][V][NC];
// masses: host [nsys].  Blocks until done.
template <class OpF>
int run_inner_apply(const Geom& g, const OpF& opf, const double2* in, double2* out, int nsys, const double* masses,
                    double r, int dagger, cudaStream_t st) {
  constexpr int NC = OpF::NC;
  using VF = typename OpF::Vec;
  using VR = typename RVecOf<VF, NC>::type;
  using PU = typename VF::unit;
  const GeomBlk gb = make_blocked(g, g.shape);
  const size_t vunits = VF::sys_units(g.V), n = (size_t)g.V * NC;
  const int ntiles = (g.V + kTile - 1) / kTile, pstride = kWarps * ntiles;
  const int nsp = pt_systems<VF>(nsys);
  const size_t bytes = 2 * align_up(sizeof(PU) * vunits * nsp) + align_up(sizeof(float2) * n * nsys) +
                       align_up(sizeof(SysState) * nsys) + align_up(sizeof(double) * pstride * nsys) +
                       align_up(sizeof(unsigned) * nsys);
  DevMem mem;
  if (!mem.alloc(bytes, st)) return SW_ERR_OOM;
  char* c = mem.as<char>();
  auto take = [&](size_t b) {
    void* p = c;
    c += align_up(b);
    return p;
  };
  const VF fp{static_cast<PU*>(take(sizeof(PU) * vunits * nsp)), g.V};
  const VF ft{static_cast<PU*>(take(sizeof(PU) * vunits * nsp)), g.V};
  const VR fr{static_cast<typename VR::unit*>(take(sizeof(float2) * n * nsys)), g.V};
  const size_t runits = VR::sys_units(g.V);
  SysState* S = static_cast<SysState*>(take(sizeof(SysState) * nsys));
  double* partials = static_cast<double*>(take(sizeof(double) * pstride * nsys));
  unsigned* tickets = static_cast<unsigned*>(take(sizeof(unsigned) * nsys));
  std::vector<SysState> hs(nsys);
  for (int i = 0; i < nsys; ++i) {
    hs[i] = SysState{};
    hs[i].mass = masses[i];
    hs[i].rr = 1.0;
    hs[i].alpha = -1.0;
    hs[i].max_iter = 1 << 30;
    hs[i].status = ST_ADMIT;
  }
  cudaMemcpyAsync(S, hs.data(), sizeof(SysState) * nsys, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nsys, st);
  cudaMemsetAsync(fr.p, 0, sizeof(float2) * n * nsys, st);
  const int gv = grid_for((const void*)demote_chi<NC, VF>, 256, g.V, nsys, ntiles);
  demote_chi<NC, VF><<<dim3(gv, nsys), 256, 0, st>>>(gb, in, dagger ? ft : fp, n, vunits, S);
  set_status<<<(nsys + 127) / 128, 128, 0, st>>>(nsys, S, ST_RUNNING);
  const RedBuf rb{partials, tickets, pstride, nullptr};
  const BatchParams bp{r, runits, n, vunits};
  const int ns = param_ns(NC);
  auto launch = [&](auto nsc) {
    constexpr int NS = decltype(nsc)::value;
    const int ngrp = (nsys + NS - 1) / NS;
    if (!dagger) {
      const int gx = grid_for((const void*)cg_k1<float, OpF, NS, GeomBlk>, kTile, g.V, ngrp, ntiles);
      cg_k1<float, OpF, NS, GeomBlk><<<dim3(gx, ngrp), kTile, 0, st>>>(gb, opf, fp, ft, bp, nsys, S, rb, nullptr, 0);
    } else {
      const int gx = grid_for((const void*)cg_k2<float, OpF, NS, VR, GeomBlk>, kTile, g.V, ngrp, ntiles);
      cg_k2<float, OpF, NS, VR, GeomBlk><<<dim3(gx, ngrp), kTile, 0, st>>>(gb, opf, ft, fr, bp, nsys, S, rb,
                                                                          nullptr, 0);
    }
  };
  if (ns == 2) launch(std::integral_constant<int, 2>{});
  else if (ns == 4) launch(std::integral_constant<int, 4>{});
  else launch(std::integral_constant<int, 1>{});
  if (!dagger) promote_vec<NC, VF><<<dim3(gv, nsys), 256, 0, st>>>(gb, ft, vunits, out, n);
  else promote_vec<NC, VR><<<dim3(gv, nsys), 256, 0, st>>>(gb, fr, runits, out, n);
  note_launches(5);
  if (const cudaError_t e = cudaStreamSynchronize(st); e != cudaSuccess) return cuda_fail(e);
  if (const cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e);
  return SW_OK;
}

}  // namespace swc
