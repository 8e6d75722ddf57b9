// Serving entry points (acopf_server_*): a request loop over resident models
// with admission by device-memory budget and continuous batching.
//
// One server thread owns the streams, the memory pool and every CUDA call of
// the loop; client threads only queue requests and read their records
// under the mutex.  A request's device region is allocated and its inputs
// uploaded on a copy stream, so that a large upload does not hold up the
// calls of the requests already running on the compute stream; a request
// takes part in ticks (or, in FIFO mode, the compute stream waits for it)
// once its upload has completed.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "host_internal.h"

using acopf::cuda_fail;
using acopf::DeviceScope;
using acopf::fail;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxInflightLimit = 16;  // upper bound of ACOPF_SERVE_OPT_INFLIGHT
constexpr int kRing = kMaxInflightLimit + 1;
// Default work of one tick (sum over its requests of buses + branches +
// generators of one call): a 20,000-bus call, or many small ones; larger
// requests run alone in their ticks.
constexpr int64_t kDefaultTickWork = 60000;

enum class St { Queued, Active, Draining, Done };

// Device region of one request: scratch, input point sets, loads, outputs.
struct ReqPlan {
  acopf::WorkspacePlan ws;
  size_t o_ws = 0, o_x = 0, o_y = 0, o_sx = 0, o_ss = 0, o_pd = 0, o_qd = 0;
  size_t o_f = 0, o_grad = 0, o_cons = 0, o_j = 0, o_h = 0, o_k = 0, bytes = 0;
};

ReqPlan plan_request(const acopf_request& r, const acopf::Layout& L) {
  ReqPlan p;
  acopf::ArenaPlan a;
  const size_t np = size_t(r.n_points), n = size_t(L.n), m = size_t(L.m);
  p.ws = acopf::workspace_plan(L);
  p.o_ws = a.take<char>(p.ws.bytes);
  p.o_x = a.take<double>(np * n);
  p.o_y = a.take<double>(np * m);
  p.o_sx = a.take<double>(np * n);
  p.o_ss = a.take<double>(np * m);
  if (r.Pd) {
    p.o_pd = a.take<double>(size_t(L.nb));
    p.o_qd = a.take<double>(size_t(L.nb));
  }
  p.o_f = a.take<double>(size_t(r.n_calls));
  p.o_grad = a.take<double>(n);
  p.o_cons = a.take<double>(m);
  p.o_j = a.take<double>(size_t(L.nnzj));
  p.o_h = a.take<double>(size_t(L.nnzh));
  p.o_k = a.take<double>(size_t(L.nnzk));
  p.bytes = a.off;
  return p;
}

struct Req {
  uint64_t id = 0;
  acopf_request r{};
  acopf::Layout L;
  ReqPlan plan;
  St st = St::Queued;         // server thread
  bool admitted = false;      // under the mutex
  bool done = false;          // under the mutex
  acopf_status result = ACOPF_OK;
  Clock::time_point t_submit, t_admit, t_done;
  // server-thread state
  char* mem = nullptr;
  acopf::DevModel dm{};
  int32_t issued = 0;
  int variant = 0;
  cudaEvent_t done_ev = nullptr;
  cudaEvent_t ready_ev = nullptr;  // its inputs are on the device (copy stream)
  bool ready = false;
  std::vector<int4> items1, items2;  // instance index 0; patched per tick

  double* dev(size_t off) const { return reinterpret_cast<double*>(mem + off); }
  acopf::EvalArgs args(int32_t call) const {
    acopf::EvalArgs a;
    std::memset(&a, 0, sizeof(a));
    const size_t k = size_t(call % r.n_points), n = size_t(L.n), m = size_t(L.m);
    a.x = dev(plan.o_x) + k * n;
    a.y = dev(plan.o_y) + k * m;
    a.sigma_x = dev(plan.o_sx) + k * n;
    a.sigma_s = dev(plan.o_ss) + k * m;
    a.obj_weight = r.obj_weight;
    a.delta_w = r.delta_w;
    a.delta_c = r.delta_c;
    a.f = dev(plan.o_f) + call;
    a.grad = dev(plan.o_grad);
    a.cons = dev(plan.o_cons);
    a.jvals = dev(plan.o_j);
    a.hvals = dev(plan.o_h);
    a.kvals = dev(plan.o_k);
    return a;
  }
};

// One slot of the tick tables: [DevModel x A][EvalArgs x A][items], in
// page-locked host memory and on the device.
struct Slot {
  char* host = nullptr;
  char* dev = nullptr;
  size_t cap = 0;
  cudaEvent_t ev = nullptr;
  bool busy = false;
};

}  // namespace

struct acopf_server {
  int device = 0;
  int64_t budget = 0;
  int32_t mode = ACOPF_SERVE_CONTINUOUS;
  int32_t max_active = 1;
  std::atomic<int> max_inflight{16};  // ticks in flight (continuous mode)
  std::atomic<int64_t> tick_work{kDefaultTickWork};  // work of one tick (continuous mode)
  cudaStream_t stream = nullptr;       // calls, tick tables, output copies
  cudaStream_t copy_stream = nullptr;  // request regions: allocation, inputs, release
  cudaMemPool_t pool = nullptr;
  std::thread th;
  // guarded by mu
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<Req*> queue;
  std::map<uint64_t, Req*> reqs;
  acopf_server_stats stats{};
  // server thread only
  std::vector<Req*> active;
  Slot ring[kRing];
  int ring_next = 0;
  std::deque<int> inflight;
};

namespace {

double seconds(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

// Marks a request done (under the lock) and wakes its waiters.
void complete(acopf_server* S, Req* q, acopf_status st) {
  std::lock_guard<std::mutex> lk(S->mu);
  q->st = St::Done;
  q->done = true;
  q->result = st;
  q->t_done = Clock::now();
  S->stats.completed++;
  if (q->admitted) {
    S->stats.bytes_in_use -= int64_t(q->plan.bytes);
    S->stats.active--;
  }
  S->cv_done.notify_all();
}

// Copies the request's outputs to its host buffers and marks its end.
cudaError_t finish_request(acopf_server* S, Req* q) {
  const acopf_request& r = q->r;
  const acopf::Layout& L = q->L;
  cudaError_t e = cudaSuccess;
  auto d2h = [&](double* host, size_t off, size_t count) {
    if (host && count && e == cudaSuccess)
      e = cudaMemcpyAsync(host, q->dev(off), count * sizeof(double), cudaMemcpyDeviceToHost,
                          S->stream);
  };
  d2h(r.f_calls, q->plan.o_f, size_t(r.n_calls));
  d2h(r.grad, q->plan.o_grad, size_t(L.n));
  d2h(r.cons, q->plan.o_cons, size_t(L.m));
  d2h(r.jvals, q->plan.o_j, size_t(L.nnzj));
  d2h(r.hvals, q->plan.o_h, size_t(L.nnzh));
  d2h(r.kvals, q->plan.o_k, size_t(L.nnzk));
  if (e == cudaSuccess) e = cudaEventRecord(q->done_ev, S->stream);
  q->st = St::Draining;
  return e;
}

// Allocates and fills the request's device region; in FIFO mode also
// queues all its calls as single-instance launches.
cudaError_t start_request(acopf_server* S, Req* q) {
  const acopf_request& r = q->r;
  const acopf::Layout& L = q->L;
  const ReqPlan& p = q->plan;
  void* mem = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&mem, p.bytes, S->pool, S->copy_stream);
  if (e != cudaSuccess) return e;
  q->mem = static_cast<char*>(mem);
  e = cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ready_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(q->mem + p.o_ws, 0, p.ws.bytes, S->copy_stream);  // arrival counter = 0
  auto h2d = [&](size_t off, const double* src, size_t count) {
    if (e == cudaSuccess && count)
      e = cudaMemcpyAsync(q->dev(off), src, count * sizeof(double), cudaMemcpyHostToDevice,
                          S->copy_stream);
  };
  const size_t np = size_t(r.n_points);
  h2d(p.o_x, r.x, np * size_t(L.n));
  h2d(p.o_y, r.y, np * size_t(L.m));
  h2d(p.o_sx, r.sigma_x, np * size_t(L.n));
  h2d(p.o_ss, r.sigma_s, np * size_t(L.m));
  if (r.Pd) {
    h2d(p.o_pd, r.Pd, size_t(L.nb));
    h2d(p.o_qd, r.Qd, size_t(L.nb));
  }
  if (e == cudaSuccess) e = cudaEventRecord(q->ready_ev, S->copy_stream);
  if (e != cudaSuccess) return e;
  q->dm = r.model->dm;
  acopf::bind_workspace(q->dm, q->mem + p.o_ws, p.ws);
  if (r.Pd) {
    q->dm.Pd = q->dev(p.o_pd);
    q->dm.Qd = q->dev(p.o_qd);
  }
  q->variant = (r.delta_w != 0.0 || r.delta_c != 0.0 ? 2 : 0) + (q->dm.has_shunt ? 1 : 0);
  acopf::append_items(L, 0, q->items1, q->items2);
  if (S->mode == ACOPF_SERVE_FIFO) {  // in arrival order: the compute stream waits for it
    q->ready = true;
    e = cudaStreamWaitEvent(S->stream, q->ready_ev, 0);
    for (int32_t c = 0; c < r.n_calls && e == cudaSuccess; ++c)
      e = acopf::launch_eval(q->dm, acopf::OUT_ALL, q->args(c), S->stream);
    q->issued = r.n_calls;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stats.launches += int64_t(r.n_calls) * acopf::launches_for(acopf::OUT_ALL);
    }
    if (e == cudaSuccess) e = finish_request(S, q);
  }
  return e;
}

cudaError_t retire_slot(acopf_server* S, int k, bool wait) {
  Slot& sl = S->ring[k];
  if (!sl.busy) return cudaSuccess;
  cudaError_t e = wait ? cudaEventSynchronize(sl.ev) : cudaEventQuery(sl.ev);
  if (e == cudaErrorNotReady) return e;
  sl.busy = false;
  auto it = std::find(S->inflight.begin(), S->inflight.end(), k);
  if (it != S->inflight.end()) S->inflight.erase(it);
  return e;
}

cudaError_t grow_slot(acopf_server* S, Slot& sl, size_t need) {
  // Every tick in flight may read a slot: let them finish first.
  for (int k = 0; k < kRing; ++k) {
    cudaError_t e = retire_slot(S, k, true);
    if (e != cudaSuccess) return e;
  }
  if (sl.host) cudaFreeHost(sl.host);
  if (sl.dev) cudaFree(sl.dev);
  sl.host = sl.dev = nullptr;
  sl.cap = 0;
  const size_t cap = std::max<size_t>(need + need / 2, 1 << 16);
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&sl.host), cap, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.dev), cap);
  if (e == cudaSuccess) sl.cap = cap;
  return e;
}

// Work of one call of a request (the kernels' units: buses, branches,
// generators).
int64_t call_work(const Req* q) { return int64_t(q->L.nb) + q->L.nl + q->L.ng; }

// One continuous-batching step: one call each of the runnable requests
// (admitted, inputs on the device, calls left) chosen for this tick, in one
// batched evaluation.  The longest-admitted runnable request always takes
// part (so every request progresses); the others join in order of least
// remaining work (calls left x work per call; ties: arrival) while the
// tick's work stays within the budget.  A small request thus shares its
// ticks with other small ones instead of waiting behind every large one.
cudaError_t tick(acopf_server* S) {
  std::vector<Req*> cand;
  for (Req* q : S->active)
    if (q->st == St::Active && q->ready && q->issued < q->r.n_calls) cand.push_back(q);
  if (cand.empty()) return cudaSuccess;
  auto oldest = std::min_element(cand.begin(), cand.end(),
                                 [](const Req* a, const Req* b) { return a->id < b->id; });
  std::iter_swap(cand.begin(), oldest);
  std::sort(cand.begin() + 1, cand.end(), [](const Req* a, const Req* b) {
    const int64_t wa = call_work(a) * (a->r.n_calls - a->issued);
    const int64_t wb = call_work(b) * (b->r.n_calls - b->issued);
    return wa != wb ? wa < wb : a->id < b->id;
  });
  std::vector<Req*> members{cand.front()};
  int64_t work = call_work(cand.front());
  const int64_t budget = S->tick_work.load();
  for (size_t j = 1; j < cand.size(); ++j)
    if (work + call_work(cand[j]) <= budget) {
      members.push_back(cand[j]);
      work += call_work(cand[j]);
    }
  const size_t A = members.size();
  if (A == 1) {  // a lone request runs its plain single-instance launches (same results)
    const int k = S->ring_next;
    Slot& sl = S->ring[k];
    cudaError_t e = retire_slot(S, k, true);
    Req* q = members.front();
    if (e == cudaSuccess) e = acopf::launch_eval(q->dm, acopf::OUT_ALL, q->args(q->issued), S->stream);
    if (e != cudaSuccess) return e;
    if (++q->issued == q->r.n_calls) {
      e = finish_request(S, q);
      if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(sl.ev, S->stream);
    if (e != cudaSuccess) return e;
    sl.busy = true;
    S->inflight.push_back(k);
    S->ring_next = (k + 1) % kRing;
    std::lock_guard<std::mutex> lk(S->mu);
    S->stats.ticks++;
    S->stats.launches += acopf::launches_for(acopf::OUT_ALL);
    return cudaSuccess;
  }
  size_t n1 = 0, n2 = 0;
  for (Req* q : members) {
    n1 += q->items1.size();
    n2 += q->items2.size();
  }
  const size_t o_models = 0;
  const size_t o_args = acopf::align_up(A * sizeof(acopf::DevModel), 256);
  const size_t o_items = o_args + acopf::align_up(A * sizeof(acopf::EvalArgs), 256);
  const size_t need = o_items + (n1 + n2) * sizeof(int4);
  const int k = S->ring_next;
  Slot& sl = S->ring[k];
  cudaError_t e = retire_slot(S, k, true);
  if (e != cudaSuccess) return e;
  if (need > sl.cap) {
    e = grow_slot(S, sl, need);
    if (e != cudaSuccess) return e;
  }
  auto* dmodels = reinterpret_cast<acopf::DevModel*>(sl.host + o_models);
  auto* dargs = reinterpret_cast<acopf::EvalArgs*>(sl.host + o_args);
  auto* items = reinterpret_cast<int4*>(sl.host + o_items);
  int64_t seg1[5];
  size_t w = 0;
  int variants = 0;
  for (int c = 0; c < 4; ++c) {
    seg1[c] = int64_t(w);
    for (size_t j = 0; j < A; ++j) {
      if (members[j]->variant != c) continue;
      for (int4 it : members[j]->items1) {
        it.x = int(j);
        items[w++] = it;
      }
    }
    if (int64_t(w) > seg1[c]) variants++;
  }
  seg1[4] = int64_t(w);
  for (size_t j = 0; j < A; ++j) {
    dmodels[j] = members[j]->dm;
    dargs[j] = members[j]->args(members[j]->issued);
    for (int4 it : members[j]->items2) {
      it.x = int(j);
      items[w++] = it;
    }
  }
  e = cudaMemcpyAsync(sl.dev, sl.host, need, cudaMemcpyHostToDevice, S->stream);
  if (e != cudaSuccess) return e;
  const auto* d_items = reinterpret_cast<const int4*>(sl.dev + o_items);
  e = acopf::launch_batch(reinterpret_cast<const acopf::DevModel*>(sl.dev + o_models),
                          reinterpret_cast<const acopf::EvalArgs*>(sl.dev + o_args), d_items, seg1,
                          INT32_MAX, d_items + n1, int(n2), int(n2), true, S->stream);
  if (e != cudaSuccess) return e;
  for (Req* q : members) {
    q->issued++;
    if (q->issued == q->r.n_calls) {
      e = finish_request(S, q);
      if (e != cudaSuccess) return e;
    }
  }
  e = cudaEventRecord(sl.ev, S->stream);
  if (e != cudaSuccess) return e;
  sl.busy = true;
  S->inflight.push_back(k);
  S->ring_next = (k + 1) % kRing;
  std::lock_guard<std::mutex> lk(S->mu);
  S->stats.ticks++;
  S->stats.launches += variants + (n2 > 0 ? 1 : 0);
  return cudaSuccess;
}

// Completes the requests whose last copy has finished; returns how many.
int poll_done(acopf_server* S, cudaError_t& err) {
  int done = 0;
  for (size_t i = 0; i < S->active.size();) {
    Req* q = S->active[i];
    if (q->st != St::Draining) {
      ++i;
      continue;
    }
    cudaError_t e = cudaEventQuery(q->done_ev);
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (e != cudaSuccess) err = e;
    // every use of the region is complete (the host saw its last event):
    // it goes back to the pool in the copy stream's order, where the next
    // regions are allocated
    cudaFreeAsync(q->mem, S->copy_stream);
    q->mem = nullptr;
    complete(S, q, e == cudaSuccess ? ACOPF_OK : ACOPF_E_CUDA);
    S->active.erase(S->active.begin() + long(i));
    ++done;
  }
  return done;
}

// Ends every admitted request with `st` after a CUDA failure of the loop.
void fail_all(acopf_server* S, acopf_status st) {
  cudaStreamSynchronize(S->stream);
  cudaStreamSynchronize(S->copy_stream);
  for (Req* q : S->active) {
    if (q->mem) cudaFreeAsync(q->mem, S->copy_stream);
    q->mem = nullptr;
    complete(S, q, st);
  }
  S->active.clear();
  for (int k = 0; k < kRing; ++k) S->ring[k].busy = false;
  S->inflight.clear();
}

void serve(acopf_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Req*> admitted;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (!S->queue.empty()) {
        Req* q = S->queue.front();
        if (S->stop) {  // queued requests are not started once the server stops
          S->queue.pop_front();
          q->st = St::Done;
          q->done = true;
          q->result = ACOPF_E_BUSY;
          q->t_done = Clock::now();
          S->stats.completed++;
          continue;
        }
        if (S->stats.active >= S->max_active ||
            S->stats.bytes_in_use + int64_t(q->plan.bytes) > S->budget)
          break;
        S->queue.pop_front();
        q->st = St::Active;
        q->admitted = true;
        q->t_admit = Clock::now();
        S->stats.bytes_in_use += int64_t(q->plan.bytes);
        S->stats.peak_bytes = std::max(S->stats.peak_bytes, S->stats.bytes_in_use);
        S->stats.active++;
        S->stats.peak_active = std::max(S->stats.peak_active, S->stats.active);
        admitted.push_back(q);
      }
      S->stats.queued = int32_t(S->queue.size());
      if (admitted.empty() && S->active.empty() && S->inflight.empty()) {
        if (S->stop) break;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    cudaError_t err = cudaSuccess;
    for (Req* q : admitted) {
      cudaError_t e = start_request(S, q);
      if (e == cudaErrorMemoryAllocation) {  // the pool could not serve it: this request fails
        cudaGetLastError();
        if (q->mem) cudaFreeAsync(q->mem, S->copy_stream);
        q->mem = nullptr;
        acopf::set_last_error("server: device allocation failed for a request");
        complete(S, q, ACOPF_E_OOM);
        continue;
      }
      S->active.push_back(q);
      if (e != cudaSuccess && err == cudaSuccess) err = e;
    }
    bool progressed = !admitted.empty();
    for (Req* q : S->active) {  // uploads that have completed
      if (q->ready || q->st != St::Active || err != cudaSuccess) continue;
      const cudaError_t e = cudaEventQuery(q->ready_ev);
      if (e == cudaSuccess) {
        q->ready = true;
        progressed = true;
      } else if (e != cudaErrorNotReady) {
        err = e;
      }
    }
    if (err == cudaSuccess && S->mode == ACOPF_SERVE_CONTINUOUS) {
      bool calls_left = false;
      for (Req* q : S->active)
        calls_left |= q->st == St::Active && q->ready && q->issued < q->r.n_calls;
      if (calls_left && int(S->inflight.size()) < S->max_inflight.load()) {
        err = tick(S);
        progressed = true;
      } else if (!S->inflight.empty()) {
        err = retire_slot(S, S->inflight.front(), true);
        progressed = true;
      }
    }
    while (err == cudaSuccess && !S->inflight.empty()) {  // retire finished ticks
      cudaError_t e = retire_slot(S, S->inflight.front(), false);
      if (e == cudaErrorNotReady) break;
      err = e;
    }
    if (err == cudaSuccess && poll_done(S, err) > 0) progressed = true;
    if (err != cudaSuccess) {
      acopf::set_last_error(std::string("server loop: ") + cudaGetErrorString(err));
      fail_all(S, ACOPF_E_CUDA);
      continue;
    }
    if (!progressed) {  // only copies in flight: wait briefly, or for a new request
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

Req* find(acopf_server* S, uint64_t ticket) {
  auto it = S->reqs.find(ticket);
  return it == S->reqs.end() ? nullptr : it->second;
}

void free_server(acopf_server* S) {
  for (int k = 0; k < kRing; ++k) {
    Slot& sl = S->ring[k];
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.dev) cudaFree(sl.dev);
  }
  for (auto& kv : S->reqs) {
    if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    if (kv.second->ready_ev) cudaEventDestroy(kv.second->ready_ev);
    delete kv.second;
  }
  if (S->pool) cudaMemPoolDestroy(S->pool);
  if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // namespace

extern "C" {

acopf_status acopf_server_create(int device, int64_t budget_bytes, int32_t mode,
                                 int32_t max_active, acopf_server** out) {
  if (!out) return fail(ACOPF_E_INVALID_ARG, "acopf_server_create: null output pointer");
  *out = nullptr;
  if (device < 0) return fail(ACOPF_E_NO_DEVICE, "acopf_server_create: needs a device");
  if (budget_bytes <= 0) return fail(ACOPF_E_INVALID_ARG, "acopf_server_create: budget must be > 0");
  if (mode != ACOPF_SERVE_CONTINUOUS && mode != ACOPF_SERVE_FIFO)
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_create: unknown mode");
  if (max_active < 1) return fail(ACOPF_E_INVALID_ARG, "acopf_server_create: max_active must be >= 1");
  acopf_server* S = new (std::nothrow) acopf_server;
  if (!S) return fail(ACOPF_E_OOM, "host allocation failed");
  S->device = device;
  S->budget = budget_bytes;
  S->mode = mode;
  S->max_active = max_active;
  DeviceScope ds(device);
  cudaError_t e = ds.error();
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&S->pool, &props);
    if (e != cudaSuccess) S->pool = nullptr;
  }
  if (e == cudaSuccess) {  // keep freed memory in the pool for the next requests
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  for (int k = 0; k < kRing && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&S->ring[k].ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_server(S);
    return cuda_fail(e, "acopf_server_create");
  }
  try {
    S->th = std::thread(serve, S);
  } catch (...) {
    free_server(S);
    return fail(ACOPF_E_OOM, "acopf_server_create: cannot start the server thread");
  }
  *out = S;
  return ACOPF_OK;
}

acopf_status acopf_server_destroy(acopf_server* server) {
  if (!server) return ACOPF_OK;
  {
    std::lock_guard<std::mutex> lk(server->mu);
    server->stop = true;
  }
  server->cv_work.notify_all();
  if (server->th.joinable()) server->th.join();
  DeviceScope ds(server->device);
  cudaStreamSynchronize(server->stream);
  cudaStreamSynchronize(server->copy_stream);
  free_server(server);
  return ACOPF_OK;
}

acopf_status acopf_server_submit(acopf_server* server, const acopf_request* req,
                                 uint64_t* ticket) {
  if (!server || !req || !ticket) return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: null pointer");
  const acopf_request& r = *req;
  if (!r.model) return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: null model");
  if (r.model->device != server->device)
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: model is not on the server's device");
  if (r.n_calls < 1 || r.n_points < 1)
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: n_calls and n_points must be >= 1");
  if (!r.x || !r.y || !r.sigma_x || !r.sigma_s)
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: null input");
  if ((r.Pd == nullptr) != (r.Qd == nullptr))
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_submit: give both Pd and Qd, or neither");
  acopf_status st = acopf::check_eval_scalars(r.obj_weight, r.delta_w, r.delta_c);
  if (st != ACOPF_OK) return st;
  Req* q = new (std::nothrow) Req;
  if (!q) return fail(ACOPF_E_OOM, "host allocation failed");
  q->r = r;
  q->L = r.model->hm.L;
  q->plan = plan_request(r, q->L);
  if (int64_t(q->plan.bytes) > server->budget) {
    delete q;
    return fail(ACOPF_E_BUDGET, "acopf_server_submit: the request alone exceeds the budget");
  }
  {
    std::lock_guard<std::mutex> lk(server->mu);
    if (server->stop) {
      delete q;
      return fail(ACOPF_E_BUSY, "acopf_server_submit: server is stopping");
    }
    q->id = server->next_id++;
    q->t_submit = Clock::now();
    server->reqs[q->id] = q;
    server->queue.push_back(q);
    server->stats.submitted++;
    server->stats.queued = int32_t(server->queue.size());
    *ticket = q->id;
  }
  server->cv_work.notify_all();
  return ACOPF_OK;
}

acopf_status acopf_server_poll(acopf_server* server, uint64_t ticket, int32_t* done,
                               acopf_status* result) {
  if (!server || !done) return fail(ACOPF_E_INVALID_ARG, "acopf_server_poll: null pointer");
  std::lock_guard<std::mutex> lk(server->mu);
  Req* q = find(server, ticket);
  if (!q) return fail(ACOPF_E_INVALID_ARG, "acopf_server_poll: unknown ticket");
  *done = q->done ? 1 : 0;
  if (result) *result = q->done ? q->result : ACOPF_OK;
  return ACOPF_OK;
}

acopf_status acopf_server_wait(acopf_server* server, uint64_t ticket, double timeout_s,
                               acopf_status* result) {
  if (!server) return fail(ACOPF_E_INVALID_ARG, "acopf_server_wait: null server");
  if (!(timeout_s >= 0.0) || !std::isfinite(timeout_s))
    return fail(ACOPF_E_INVALID_ARG, "acopf_server_wait: timeout must be finite and >= 0");
  std::unique_lock<std::mutex> lk(server->mu);
  Req* q = find(server, ticket);
  if (!q) return fail(ACOPF_E_INVALID_ARG, "acopf_server_wait: unknown ticket");
  const auto deadline =
      Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  if (!server->cv_done.wait_until(lk, deadline, [q] { return q->done; }))
    return fail(ACOPF_E_TIMEOUT, "acopf_server_wait: request not done within the timeout");
  if (result) *result = q->result;
  return ACOPF_OK;
}

acopf_status acopf_server_request_times(acopf_server* server, uint64_t ticket, double* admitted_s,
                                        double* done_s) {
  if (!server) return fail(ACOPF_E_INVALID_ARG, "acopf_server_request_times: null server");
  std::lock_guard<std::mutex> lk(server->mu);
  Req* q = find(server, ticket);
  if (!q) return fail(ACOPF_E_INVALID_ARG, "acopf_server_request_times: unknown ticket");
  if (!q->done) return fail(ACOPF_E_BUSY, "acopf_server_request_times: request not done");
  if (admitted_s) *admitted_s = q->admitted ? seconds(q->t_admit - q->t_submit) : -1.0;
  if (done_s) *done_s = seconds(q->t_done - q->t_submit);
  return ACOPF_OK;
}

acopf_status acopf_server_release(acopf_server* server, uint64_t ticket) {
  if (!server) return fail(ACOPF_E_INVALID_ARG, "acopf_server_release: null server");
  std::lock_guard<std::mutex> lk(server->mu);
  Req* q = find(server, ticket);
  if (!q) return fail(ACOPF_E_INVALID_ARG, "acopf_server_release: unknown ticket");
  if (!q->done) return fail(ACOPF_E_BUSY, "acopf_server_release: request not done");
  if (q->done_ev || q->ready_ev) {
    DeviceScope ds(server->device);
    if (q->done_ev) cudaEventDestroy(q->done_ev);
    if (q->ready_ev) cudaEventDestroy(q->ready_ev);
  }
  server->reqs.erase(ticket);
  delete q;
  return ACOPF_OK;
}

acopf_status acopf_server_set_option(acopf_server* server, int32_t option, int64_t value) {
  if (!server) return fail(ACOPF_E_INVALID_ARG, "acopf_server_set_option: null server");
  if (option == ACOPF_SERVE_OPT_INFLIGHT) {
    if (value < 1 || value > kMaxInflightLimit)
      return fail(ACOPF_E_INVALID_ARG, "acopf_server_set_option: in-flight ticks must be in [1, 16]");
    server->max_inflight.store(int(value));
    server->cv_work.notify_all();
    return ACOPF_OK;
  }
  if (option == ACOPF_SERVE_OPT_TICK_WORK) {
    if (value < 1)
      return fail(ACOPF_E_INVALID_ARG, "acopf_server_set_option: the tick work must be >= 1");
    server->tick_work.store(value);
    return ACOPF_OK;
  }
  return fail(ACOPF_E_INVALID_ARG, "acopf_server_set_option: unknown option");
}

acopf_status acopf_server_get_stats(acopf_server* server, acopf_server_stats* out) {
  if (!server || !out) return fail(ACOPF_E_INVALID_ARG, "acopf_server_get_stats: null pointer");
  std::lock_guard<std::mutex> lk(server->mu);
  *out = server->stats;
  return ACOPF_OK;
}

}  // extern "C"
