// Continuous-batching solve server.
//
// The server keeps gauge fields resident on the device, one Engine per field
// (lattice, operator, r, precision), each with a fixed number of system slots
// and its own CUDA stream.  A scheduler thread loops over the engines: when an
// engine's round has landed it reports the systems that finished (their
// solutions are copied to the caller's host buffers on the engine's stream),
// refills free slots from the engine's FIFO of waiting requests, and issues the
// next round.  Requests that arrive while others are on the GPU therefore join
// as slots free up, and the engines' streams overlap on the device.  A system's
// arithmetic does not depend on the other slots (per-slot scalars and
// reductions in a fixed order), so each result is bit-identical alone and in
// any mix.
//
// Admission by memory.  Gauge fields are resident (sw_server_add_field), and a
// request names a field, an operator, r and a precision: the scheduler finds
// the engine of that combination or creates it when the device-memory budget
// allows, first retiring engines it created that have gone idle (least
// recently used first); while the memory is not there the request waits,
// and requests behind it whose engines exist go ahead.  Every engine's device
// memory (packed copies, slot vectors, workspace; the links too for engines
// added with sw_server_add_engine, which are never retired) is charged
// against the budget.  Inside an engine a request waits in the engine's queue
// until a slot is free.
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

#include "driver.cuh"

namespace swc {

namespace {

struct Request {
  long long id;
  const void* chi_host;
  void* x_host;
  double mass, tol;
  int max_iter;
  std::chrono::steady_clock::time_point t_submit;
};

struct Done {
  long long id;
  sw_solve_info info;
};

// Type-erased engine with the memory it owns.
struct EngineBase {
  virtual ~EngineBase() = default;
  virtual int cap() const = 0;
  virtual size_t slot_bytes() const = 0;
  virtual double2* chi_slot(int i) = 0;
  virtual double2* x_slot(int i) = 0;
  virtual void stage(int i, double mass, double tol, int max_iter) = 0;
  virtual void issue() = 0;
  virtual bool ready() const = 0;
  virtual int complete() = 0;
  virtual void finished(std::vector<int>& out) = 0;
  virtual const SysState& state(int i) const = 0;
  virtual const double* hist() const = 0;  // device [cap][kHist][2]
  virtual cudaStream_t stream() const = 0;
  virtual int precision() const = 0;
  virtual void flush_profile() = 0;
};

template <class OpD, class OpF, bool MIXED>
struct EngineImpl : EngineBase {
  std::vector<DevMem*> owned;
  SysState* hs = nullptr;  // pinned [2 cap]
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int prec;
  std::unique_ptr<Engine<OpD, OpF, MIXED>> e;
  ~EngineImpl() override {
    if (st) cudaStreamSynchronize(st);
    e.reset();
    for (DevMem* m : owned) delete m;
    if (hs) cudaFreeHost(hs);
    if (ev) cudaEventDestroy(ev);
    if (st) cudaStreamDestroy(st);
  }
  int cap() const override { return e->cap(); }
  size_t slot_bytes() const override { return e->slot_elems() * sizeof(double2); }
  double2* chi_slot(int i) override { return e->chi_slot(i); }
  double2* x_slot(int i) override { return e->x_slot(i); }
  void stage(int i, double m, double tol, int mi) override { e->stage(i, m, tol, mi); }
  void issue() override { e->issue(); }
  bool ready() const override { return e->ready(); }
  int complete() override { return e->complete(); }
  void finished(std::vector<int>& out) override { e->finished(out); }
  const SysState& state(int i) const override { return e->state(i); }
  const double* hist() const override { return e->hist(); }
  cudaStream_t stream() const override { return st; }
  int precision() const override { return prec; }
  void flush_profile() override { e->flush_profile(); }
};

using SW64 = SWOp<double, GaugeC64, TransC64, VecC64>;
using SW32 = SWOp<float, GaugeP32, TransP32, VecP32x2>;
using SW16 = SWOp<float, GaugeP16, TransP16, VecP16>;
template <bool R1> using W64 = WOp<double, GaugeC64, VecC64, R1>;
template <bool R1> using W32 = WOp<float, GaugeP32, VecP32q, R1>;
using W32L = WOp<float, GaugeP32, VecP32q, true, true>;  // the lean r = 1 form (wilson_lean lattices)
template <bool R1> using W16 = WOp<float, GaugeP16, VecP16, R1>;

// Allocate on `st`, remembering the block for the engine's destructor.
static void* own(std::vector<DevMem*>& owned, size_t bytes, cudaStream_t st) {
  DevMem* m = new DevMem();
  if (!m->alloc(bytes, st)) {
    delete m;
    return nullptr;
  }
  owned.push_back(m);
  return m->p;
}

template <class OpD, class OpF, bool MIXED, class MakeOps>
static int build_engine(const Geom& g, int cap, double r, int prec, MakeOps make_ops,
                        std::unique_ptr<EngineBase>* out) {
  auto impl = std::make_unique<EngineImpl<OpD, OpF, MIXED>>();
  impl->prec = prec;
  if (cudaStreamCreateWithFlags(&impl->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&impl->ev, cudaEventDisableTiming) != cudaSuccess)
    return SW_ERR_CUDA;
  OpD opd;
  OpF opf;
  if (int e = make_ops(impl->owned, impl->st, &opd, &opf)) return e;
  const size_t n = (size_t)g.V * OpD::NC;
  double2* chi = (double2*)own(impl->owned, sizeof(double2) * n * cap, impl->st);
  double2* x = (double2*)own(impl->owned, sizeof(double2) * n * cap, impl->st);
  void* wsm = own(impl->owned, workspace_bytes_for<typename OpF::Vec>(g.V, OpD::NC, cap, MIXED), impl->st);
  if (!chi || !x || !wsm) return SW_ERR_OOM;
  if (cudaMallocHost((void**)&impl->hs, sizeof(SysState) * 2 * cap) != cudaSuccess) return SW_ERR_OOM;
  const Workspace ws = carve_workspace_for<typename OpF::Vec>(wsm, g.V, OpD::NC, cap, MIXED);
  impl->e = std::make_unique<Engine<OpD, OpF, MIXED>>(g, opd, opf, r, cap, chi, x, ws, impl->hs, impl->hs + cap,
                                                      impl->st, impl->ev);
  if (const cudaError_t e = cudaStreamSynchronize(impl->st); e != cudaSuccess) return cuda_fail(e);
  *out = std::move(impl);
  return SW_OK;
}

// Device bytes an engine will hold: resident field (+ transports), packed
// FP32 copies, chi and x slots, workspace.
static size_t engine_bytes(const Geom& g, int op, int prec, int cap, bool own_links = true) {
  const size_t V = g.V;
  const int nc = op == SW_OP_WILSON ? 12 : 3;
  const bool mixed = prec != SW_PREC_F64;
  size_t b = (own_links ? V * 576 : 0) + (op == SW_OP_WILSON ? 0 : V * 1152);
  if (prec == SW_PREC_F32_RELIABLE) b += V * 288 + (op == SW_OP_WILSON ? 0 : V * 576);
  if (prec == SW_PREC_F16_RELIABLE) b += V * 96 + (op == SW_OP_WILSON ? 0 : V * 288);
  const size_t ws = prec == SW_PREC_F16_RELIABLE
                        ? workspace_bytes_pt(g.V, nc, cap, true, 4 * V * (nc + 1))
                        : workspace_bytes(g.V, nc, cap, mixed);
  b += 2 * V * nc * 16 * (size_t)cap + ws + (8u << 10) * 8;
  return b;
}

// own_links: the engine keeps its own copy of U (the caller's buffer may be
// freed after the call); otherwise U is a resident field of the server, which
// outlives the engine.
static int make_engine(const Geom& g, int op, const double2* U, double r, int prec, int cap,
                       std::unique_ptr<EngineBase>* out, bool own_links = true) {
  const size_t V = g.V;
  auto copy_links = [&](std::vector<DevMem*>& owned, cudaStream_t st, double2** Ur) -> int {
    if (!own_links) {
      *Ur = const_cast<double2*>(U);
      return SW_OK;
    }
    *Ur = (double2*)own(owned, V * 576, st);
    if (!*Ur) return SW_ERR_OOM;
    return cudaMemcpyAsync(*Ur, U, V * 576, cudaMemcpyDeviceToDevice, st) == cudaSuccess ? SW_OK : SW_ERR_CUDA;
  };
  const int gp = sm_count() * 8;
  if (op == SW_OP_STAGGERED_WILSON) {
    auto sw_common = [&](std::vector<DevMem*>& owned, cudaStream_t st, double2** Ur, double2** Wr) -> int {
      if (int e = copy_links(owned, st, Ur)) return e;
      *Wr = (double2*)own(owned, V * 1152, st);
      if (!*Wr) return SW_ERR_OOM;
      return hypercube_build_f64(g, *Ur, *Wr, st);
    };
    if (prec == SW_PREC_F64)
      return build_engine<SW64, SW64, false>(g, cap, r, prec, [&](auto& owned, cudaStream_t st, SW64* d, SW64* f) {
        double2 *Ur, *Wr;
        if (int e = sw_common(owned, st, &Ur, &Wr)) return e;
        *d = *f = SW64{GaugeC64{Ur}, TransC64{Wr}};
        return (int)SW_OK;
      }, out);
    if (prec == SW_PREC_F16_RELIABLE)
      return build_engine<SW64, SW16, true>(g, cap, r, prec, [&](auto& owned, cudaStream_t st, SW64* d, SW16* f) {
        double2 *Ur, *Wr;
        if (int e = sw_common(owned, st, &Ur, &Wr)) return e;
        if (int e = check_su3(g, Ur, st)) return e;
        __half2* u16 = (__half2*)own(owned, V * 96, st);
        __half2* w16 = (__half2*)own(owned, V * 288, st);
        if (!u16 || !w16) return (int)SW_ERR_OOM;
        pack_links_h12<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), Ur, u16);
        pack_mats_h<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 8, Wr, w16);
        note_launches(2);
        *d = SW64{GaugeC64{Ur}, TransC64{Wr}};
        *f = SW16{GaugeP16{u16}, TransP16{w16}};
        return (int)SW_OK;
      }, out);
    return build_engine<SW64, SW32, true>(g, cap, r, prec, [&](auto& owned, cudaStream_t st, SW64* d, SW32* f) {
      double2 *Ur, *Wr;
      if (int e = sw_common(owned, st, &Ur, &Wr)) return e;
      float2* u32 = (float2*)own(owned, V * 288, st);
      float2* w32 = (float2*)own(owned, V * 576, st);
      if (!u32 || !w32) return (int)SW_ERR_OOM;
      pack_mats_p32<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 4, Ur, u32);
      pack_mats_p32<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 8, Wr, w32);
      note_launches(2);
      *d = SW64{GaugeC64{Ur}, TransC64{Wr}};
      *f = SW32{GaugeP32{u32}, TransP32{w32}};
      return (int)SW_OK;
    }, out);
  }
  auto wilson = [&](auto r1) -> int {
    constexpr bool R1 = decltype(r1)::value;
    if (prec == SW_PREC_F64)
      return build_engine<W64<R1>, W64<R1>, false>(g, cap, r, prec,
                                                   [&](auto& owned, cudaStream_t st, W64<R1>* d, W64<R1>* f) {
        double2* Ur;
        if (int e = copy_links(owned, st, &Ur)) return e;
        *d = *f = W64<R1>{GaugeC64{Ur}};
        return (int)SW_OK;
      }, out);
    if (prec == SW_PREC_F16_RELIABLE)
      return build_engine<W64<R1>, W16<R1>, true>(g, cap, r, prec,
                                                  [&](auto& owned, cudaStream_t st, W64<R1>* d, W16<R1>* f) {
        double2* Ur;
        if (int e = copy_links(owned, st, &Ur)) return e;
        if (int e = check_su3(g, Ur, st)) return e;
        __half2* u16 = (__half2*)own(owned, V * 96, st);
        if (!u16) return (int)SW_ERR_OOM;
        pack_links_h12<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), Ur, u16);
        note_launches(1);
        *d = W64<R1>{GaugeC64{Ur}};
        *f = W16<R1>{GaugeP16{u16}};
        return (int)SW_OK;
      }, out);
    auto f32 = [&](auto tag) -> int {  // tag: the FP32 operator type
      using OF = typename decltype(tag)::type;
      return build_engine<W64<R1>, OF, true>(g, cap, r, prec, [&](auto& owned, cudaStream_t st, W64<R1>* d, OF* f) {
        double2* Ur;
        if (int e = copy_links(owned, st, &Ur)) return e;
        float2* u32 = (float2*)own(owned, V * 288, st);
        if (!u32) return (int)SW_ERR_OOM;
        pack_mats_p32<<<gp, 256, 0, st>>>(make_blocked(g, g.shape), 4, Ur, u32);
        note_launches(1);
        *d = W64<R1>{GaugeC64{Ur}};
        *f = OF{GaugeP32{u32}};
        return (int)SW_OK;
      }, out);
    };
    if constexpr (R1)
      if (wilson_lean(g)) return f32(std::common_type<W32L>{});
    return f32(std::common_type<W32<R1>>{});
  };
  return r == 1.0 ? wilson(std::true_type{}) : wilson(std::false_type{});
}

}  // namespace

struct Server {
  int device = 0;
  size_t budget = 0, used = 0;
  size_t fixed = 0;  // bytes of the fields and of the engines added by hand (never released while serving)
  // resident gauge fields (std::deque: references stay valid as fields are added)
  struct Field {
    Geom g;
    DevMem* mem = nullptr;
    int slots = 0;
  };
  std::deque<Field> fields;
  // the (field, operator, r, precision) an engine was created for on demand (field < 0: added by hand)
  struct Key {
    int field = -1, op = 0, prec = 0;
    double r = 1.0;
    bool operator==(const Key& o) const { return field == o.field && op == o.op && prec == o.prec && r == o.r; }
  };
  std::vector<Key> keys;
  std::vector<size_t> charged;  // bytes each engine holds against the budget
  std::vector<long long> last_used;  // scheduler pass of the engine's last work (LRU retirement)
  struct Waiting {
    Request rq;
    Key key;
    bool counted = false;
  };
  std::deque<Waiting> waiting;  // requests whose engine does not exist yet
  long long created = 0, retired = 0, waited = 0, pass = 0;
  std::vector<std::unique_ptr<EngineBase>> engines;  // nullptr: retired
  std::vector<Geom> geoms;
  std::vector<std::deque<Request>> queues;
  std::vector<std::vector<Request>> slots;  // per engine, per slot: the request it holds (id < 0: free)
  std::vector<char> in_flight;
  std::vector<char> has_work;
  struct Copy {
    cudaEvent_t ev;
    Done done;
    std::chrono::steady_clock::time_point t_submit;
  };
  std::deque<Copy> copies;
  std::vector<cudaEvent_t> event_pool;
  std::deque<Done> done;
  long long next_id = 1, outstanding = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int error = SW_OK;
  std::thread thread;

  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }

  void fail(int code) {
    std::lock_guard<std::mutex> lk(mu);
    if (error == SW_OK) error = code;
    cv_done.notify_all();
  }

  // An engine created on demand that holds no request (queued, in a slot or
  // in flight) may be retired.
  bool idle(size_t k) {
    if (!engines[k] || keys[k].field < 0 || in_flight[k] || has_work[k] || !queues[k].empty()) return false;
    for (const Request& rq : slots[k])
      if (rq.id >= 0) return false;
    return true;
  }

  // Give requests without an engine one: an existing engine of their
  // (field, operator, r, precision), else a new one if the budget allows after
  // retiring idle engines created on demand (least recently used first).  A
  // request whose engine cannot fit yet keeps waiting; the ones behind it go
  // ahead if their engines exist.  Scheduler thread only.
  bool admit_waiting() {
    bool moved = false;
    std::unique_lock<std::mutex> lk(mu);
    for (auto it = waiting.begin(); it != waiting.end();) {
      int k = -1;
      for (size_t j = 0; j < engines.size(); ++j)
        if (engines[j] && keys[j] == it->key) k = (int)j;
      if (k < 0) {
        const Field& f = fields[it->key.field];
        const size_t need = engine_bytes(f.g, it->key.op, it->key.prec, f.slots, false);
        while (used + need > budget) {  // retire the least recently used idle engine
          int victim = -1;
          for (size_t j = 0; j < engines.size(); ++j)
            if (idle(j) && (victim < 0 || last_used[j] < last_used[victim])) victim = (int)j;
          if (victim < 0) break;
          cudaStreamSynchronize(engines[victim]->stream());
          engines[victim].reset();  // its device memory goes back to the library's pool
          used -= charged[victim];
          charged[victim] = 0;
          ++retired;
        }
        if (used + need > budget) {  // not yet: wait for memory
          if (!it->counted) {
            it->counted = true;
            ++waited;
          }
          ++it;
          continue;
        }
        std::unique_ptr<EngineBase> eng;
        const Key key = it->key;
        const Geom g = f.g;
        const int slots_per = f.slots;
        const double2* U = f.mem->as<double2>();
        lk.unlock();  // engine set-up allocates and waits on the device: submitters need not wait for it
        const int rc = make_engine(g, key.op, U, key.r, key.prec, slots_per, &eng, false);
        lk.lock();
        if (rc != SW_OK) {
          if (error == SW_OK) error = rc;
          cv_done.notify_all();
          return moved;
        }
        used += need;
        ++created;
        k = (int)engines.size();
        push_engine(std::move(eng), g, slots_per, key, need);
      }
      queues[k].push_back(it->rq);
      it = waiting.erase(it);
      moved = true;
    }
    return moved;
  }

  // Append an engine and its bookkeeping (caller holds mu, or serving has not started).
  void push_engine(std::unique_ptr<EngineBase> eng, const Geom& g, int nslots, const Key& key, size_t bytes) {
    engines.push_back(std::move(eng));
    geoms.push_back(g);
    queues.emplace_back();
    Request freeslot{};
    freeslot.id = -1;
    slots.emplace_back(nslots, freeslot);
    in_flight.push_back(0);
    has_work.push_back(0);
    keys.push_back(key);
    charged.push_back(bytes);
    last_used.push_back(pass);
  }

  // Scheduler thread: see the file comment.
  void loop() {
    cudaSetDevice(device);
    std::vector<int> fin;
    std::vector<double> hh(2 * kHist);
    while (true) {
      bool progressed = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
      }
      ++pass;
      if (admit_waiting()) progressed = true;
      if (error != SW_OK) return;
      for (size_t k = 0; k < engines.size(); ++k) {
        if (!engines[k]) continue;  // retired
        EngineBase& e = *engines[k];
        if (in_flight[k]) {
          if (!e.ready()) continue;
          const int act = e.complete();
          in_flight[k] = 0;
          progressed = true;
          if (act < 0) {
            fail(act);
            return;
          }
          if (prof_enabled()) {  // the stream is idle: hand timing samples to the profiler
            e.flush_profile();
            prof_flush();
          }
          has_work[k] = act > 0;
          fin.clear();
          e.finished(fin);
          for (int i : fin) {
            Request& rq = slots[k][i];
            Copy c;
            c.done.id = rq.id;
            c.t_submit = rq.t_submit;
            c.done.info = sw_solve_info{};
            cudaMemcpyAsync(hh.data(), e.hist() + (size_t)i * 2 * kHist, sizeof(double) * hh.size(),
                            cudaMemcpyDeviceToHost, e.stream());
            cudaStreamSynchronize(e.stream());
            fill_info(e.state(i), hh.data(), e.precision(), 0.0, &c.done.info);
            cudaMemcpyAsync(rq.x_host, e.x_slot(i), e.slot_bytes(), cudaMemcpyDeviceToHost, e.stream());
            c.ev = get_event();
            cudaEventRecord(c.ev, e.stream());
            copies.push_back(c);
            rq.id = -1;  // slot free; later writes to it follow the copy in stream order
          }
        }
        // refill free slots from the queue
        int admitted = 0;
        {
          std::lock_guard<std::mutex> lk(mu);
          for (int i = 0; i < e.cap() && !queues[k].empty(); ++i) {
            if (slots[k][i].id >= 0) continue;
            Request rq = queues[k].front();
            queues[k].pop_front();
            slots[k][i] = rq;
            cudaMemcpyAsync(e.chi_slot(i), rq.chi_host, e.slot_bytes(), cudaMemcpyHostToDevice, e.stream());
            cudaMemsetAsync(e.x_slot(i), 0, e.slot_bytes(), e.stream());
            e.stage(i, rq.mass, rq.tol, rq.max_iter);
            ++admitted;
          }
        }
        if (admitted || has_work[k]) {
          e.issue();
          in_flight[k] = 1;
          progressed = true;
          last_used[k] = pass;
        }
      }
      // solutions whose copies have landed
      while (!copies.empty()) {
        const cudaError_t q = cudaEventQuery(copies.front().ev);
        if (q == cudaErrorNotReady) break;
        Copy c = copies.front();
        copies.pop_front();
        event_pool.push_back(c.ev);
        if (q != cudaSuccess) {
          fail(cuda_fail(q));
          return;
        }
        c.done.info.seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - c.t_submit).count();
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(c.done);
        --outstanding;
        cv_done.notify_all();
        progressed = true;
      }
      if (!progressed) {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::microseconds(50));
      }
    }
  }
};

}  // namespace swc

using namespace swc;

struct sw_server_s {
  Server s;
};

extern "C" {

int sw_server_create(size_t hbm_budget_bytes, sw_server* out) {
  if (!out) return SW_ERR_NULL;
  *out = nullptr;
  auto* srv = new sw_server_s();
  if (cudaGetDevice(&srv->s.device) != cudaSuccess) {
    delete srv;
    return SW_ERR_CUDA;
  }
  srv->s.budget = hbm_budget_bytes;
  *out = srv;
  return SW_OK;
}

int sw_server_add_engine(sw_server srv, const sw_lattice* lat, int op, const void* U, double r, int precision,
                         int slots, int* engine) {
  if (!srv || !engine) return SW_ERR_NULL;
  Server& s = srv->s;
  if (s.thread.joinable()) return SW_ERR_ARG;  // engines are fixed once serving has started
  Geom g;
  if (int e = make_geom(lat, &g)) return e;
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON) return SW_ERR_ARG;
  if (precision != SW_PREC_F64 && precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE)
    return SW_ERR_ARG;
  if (slots < 1 || slots > 4096 || !(r == r)) return SW_ERR_ARG;
  if (int e = check_buf(U, (size_t)g.V * 576)) return e;
  const size_t need = engine_bytes(g, op, precision, slots);
  if (s.used + need > s.budget) return SW_ERR_OOM;
  std::unique_ptr<EngineBase> eng;
  if (int e = make_engine(g, op, static_cast<const double2*>(U), r, precision, slots, &eng)) return e;
  s.used += need;
  s.fixed += need;
  *engine = (int)s.engines.size();
  s.push_engine(std::move(eng), g, slots, Server::Key{}, need);
  return SW_OK;
}

int sw_server_add_field(sw_server srv, const sw_lattice* lat, const void* U, int slots, int* field) {
  if (!srv || !field) return SW_ERR_NULL;
  Server& s = srv->s;
  Geom g;
  if (int e = make_geom(lat, &g)) return e;
  if (slots < 1 || slots > 4096) return SW_ERR_ARG;
  const size_t bytes = (size_t)g.V * 576;
  if (int e = check_buf(U, bytes)) return e;
  std::lock_guard<std::mutex> lk(s.mu);
  if (s.error != SW_OK) return s.error;
  if (s.fixed + bytes > s.budget) return SW_ERR_OOM;
  // retire idle on-demand engines if the field does not fit beside them
  while (s.used + bytes > s.budget) {
    int victim = -1;
    for (size_t j = 0; j < s.engines.size(); ++j)
      if (s.idle(j) && (victim < 0 || s.last_used[j] < s.last_used[victim])) victim = (int)j;
    if (victim < 0) return SW_ERR_OOM;
    cudaStreamSynchronize(s.engines[victim]->stream());
    s.engines[victim].reset();
    s.used -= s.charged[victim];
    s.charged[victim] = 0;
    ++s.retired;
  }
  Server::Field f;
  f.g = g;
  f.slots = slots;
  f.mem = new DevMem();
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    delete f.mem;
    return SW_ERR_CUDA;
  }
  int rc = SW_OK;
  if (!f.mem->alloc(bytes, st)) rc = SW_ERR_OOM;
  else if (cudaMemcpyAsync(f.mem->p, U, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
           cudaStreamSynchronize(st) != cudaSuccess)
    rc = SW_ERR_CUDA;
  f.mem->s = nullptr;  // later frees are ordered on the legacy stream, after every engine has synchronised
  cudaStreamDestroy(st);
  if (rc != SW_OK) {
    delete f.mem;
    return rc;
  }
  s.used += bytes;
  s.fixed += bytes;
  *field = (int)s.fields.size();
  s.fields.push_back(f);
  return SW_OK;
}

int sw_server_submit_field(sw_server srv, int field, int op, double r, int precision, const void* chi_host,
                           void* x_host, double mass, double tol, int max_iter, long long* request) {
  if (!srv || !chi_host || !x_host || !request) return SW_ERR_NULL;
  Server& s = srv->s;
  if (op != SW_OP_STAGGERED_WILSON && op != SW_OP_WILSON) return SW_ERR_ARG;
  if (precision != SW_PREC_F64 && precision != SW_PREC_F32_RELIABLE && precision != SW_PREC_F16_RELIABLE)
    return SW_ERR_ARG;
  if (!(tol > 0.0 && tol < 1.0) || max_iter < 1 || !(mass == mass) || !(r == r)) return SW_ERR_ARG;
  std::lock_guard<std::mutex> lk(s.mu);
  if (s.error != SW_OK) return s.error;
  if (field < 0 || field >= (int)s.fields.size()) return SW_ERR_ARG;
  const Server::Field& f = s.fields[field];
  // a request whose engine could never fit beside the fields and the fixed engines is refused now
  if (s.fixed + engine_bytes(f.g, op, precision, f.slots, false) > s.budget) return SW_ERR_OOM;
  if (!s.thread.joinable()) s.thread = std::thread([&s] { s.loop(); });
  Server::Waiting w;
  w.rq = Request{s.next_id++, chi_host, x_host, mass, tol, max_iter, std::chrono::steady_clock::now()};
  w.key.field = field;
  w.key.op = op;
  w.key.prec = precision;
  w.key.r = r;
  s.waiting.push_back(w);
  ++s.outstanding;
  *request = w.rq.id;
  s.cv_work.notify_one();
  return SW_OK;
}

int sw_server_stats(sw_server srv, sw_server_stats_t* out) {
  if (!srv || !out) return SW_ERR_NULL;
  Server& s = srv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  int live = 0;
  for (auto& e : s.engines) live += e != nullptr;
  out->engines_live = live;
  out->engines_created = (int)s.created;
  out->engines_retired = (int)s.retired;
  out->requests_waited_for_memory = s.waited;
  out->requests_waiting = (long long)s.waiting.size();
  out->bytes_charged = s.used;
  out->budget = s.budget;
  return SW_OK;
}

int sw_server_submit(sw_server srv, int engine, const void* chi_host, void* x_host, double mass, double tol,
                     int max_iter, long long* request) {
  if (!srv || !chi_host || !x_host || !request) return SW_ERR_NULL;
  Server& s = srv->s;
  if (!(tol > 0.0 && tol < 1.0) || max_iter < 1 || !(mass == mass)) return SW_ERR_ARG;
  std::lock_guard<std::mutex> lk(s.mu);
  if (engine < 0 || engine >= (int)s.engines.size() || s.keys[engine].field >= 0) return SW_ERR_ARG;
  if (s.error != SW_OK) return s.error;
  if (!s.thread.joinable()) s.thread = std::thread([&s] { s.loop(); });
  Request rq{s.next_id++, chi_host, x_host, mass, tol, max_iter, std::chrono::steady_clock::now()};
  s.queues[engine].push_back(rq);
  ++s.outstanding;
  *request = rq.id;
  s.cv_work.notify_one();
  return SW_OK;
}

int sw_server_poll(sw_server srv, int max, long long* requests, sw_solve_info* infos, int* n_done) {
  if (!srv || !n_done || (max > 0 && (!requests || !infos))) return SW_ERR_NULL;
  Server& s = srv->s;
  std::lock_guard<std::mutex> lk(s.mu);
  int k = 0;
  while (k < max && !s.done.empty()) {
    requests[k] = s.done.front().id;
    infos[k] = s.done.front().info;
    s.done.pop_front();
    ++k;
  }
  *n_done = k;
  return s.error;
}

int sw_server_drain(sw_server srv, double timeout_s) {
  if (!srv) return SW_ERR_NULL;
  Server& s = srv->s;
  std::unique_lock<std::mutex> lk(s.mu);
  const bool ok = s.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                     [&] { return s.outstanding == 0 || s.error != SW_OK; });
  if (s.error != SW_OK) return s.error;
  return ok ? SW_OK : SW_ERR_TIMEOUT;
}

int sw_server_destroy(sw_server srv) {
  if (!srv) return SW_ERR_NULL;
  Server& s = srv->s;
  {
    std::lock_guard<std::mutex> lk(s.mu);
    s.stop = true;
    s.cv_work.notify_all();
  }
  if (s.thread.joinable()) s.thread.join();
  for (auto& e : s.engines)
    if (e) cudaStreamSynchronize(e->stream());
  for (auto& c : s.copies) cudaEventDestroy(c.ev);
  for (cudaEvent_t e : s.event_pool) cudaEventDestroy(e);
  s.engines.clear();
  for (auto& f : s.fields) delete f.mem;
  delete srv;
  return SW_OK;
}

}  // extern "C"
