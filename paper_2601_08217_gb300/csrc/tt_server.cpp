// Serving form of the channel engine: continuous batching of the slot pushes of many UEs.
//
// tt_server_start gives an engine a batching thread.  Every slot pushed through the public push
// calls (from any thread) becomes a request with its arrival time.  The thread launches whatever
// is pending as one batch (tt_engine_run) whenever fewer than max_inflight_batches are on the GPU,
// so requests that arrive while others run are admitted into the next batch and their work
// overlaps on the device (per-UE isolation, Sec. III-C, keeps every result the same alone and in
// the mix).  Each batch in flight launches on its own lane of streams, work list and counters, so
// a batch's kernels start while the previous batches' tails still run.  A push into a full ring waits for room instead of being refused.  Each batch's
// completion is stamped on the device (%globaltimer) and mapped to the host clock, so a request's
// latency does not include how soon the host noticed the completion.
//
// tt_chan_create_queued adds an admission waiting list: channels that do not fit the HBM budget
// wait, in arrival order, until destroyed channels free memory.
//
// tt_engine_serve is the load generator of the serving benchmark: Poisson slot arrivals per UE
// with jitter, committed through the same request path (zero-copy commits of IQ already resident
// in each UE's ring), with a bounded per-UE queue of arrivals waiting for ring room.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <queue>
#include <random>
#include <thread>

#include "tt_engine_impl.h"

using ttx::fail;
using ttx::now_ns;
using ttx::now_us;

struct TTServer {
  tt_server_config cfg{};
  std::thread th;
  std::thread::id tid;
  std::atomic<bool> stop{false};
  static constexpr int kRing = 4096;                 // device stamps, batch seq mod kRing
  unsigned long long *h_stamp = nullptr, *d_stamp = nullptr;  // mapped pinned memory: end stamps, then start stamps
  int64_t offset_ns = 0, calib_err_ns = 0;           // device timer - host steady clock
  int64_t count_from_ns = 0;                         // arrivals earlier than this are not counted
  struct Batch {
    uint64_t seq;
    std::vector<int64_t> arrivals;
    std::vector<tt_chan *> chans;  // the channels it launched
    cudaEvent_t done = nullptr;    // its completion event (a hint polled without the engine lock)
  };
  std::atomic<int64_t> first_pending_ns{0};           // arrival of the oldest unlaunched request, 0 = none
  int64_t coalesce_ns = 20000;
  std::deque<Batch> batches;                         // launched, not yet seen complete
  std::vector<double> lat_ns;
  uint64_t requests = 0, queued = 0, refused = 0, completed = 0, n_batches = 0, batched = 0, misses = 0;
  double gpu_ns = 0.0;                               // device time from batches' start to end stamps
  int64_t first_start = 0, last_end = 0, busy_until = 0;
  double deadline_ns = 500e3;
  tt_status err = TT_OK;
  std::string err_msg;
};

// Batches in flight by default, each on its own launch lane where the engine allows it.  At 512
// serving UEs (GPU 98% busy) p99 went 689, 575, 523 and 411-435 us with 3, 5, 6 and 8 in flight.
constexpr int kDefaultInflight = 8;

namespace ttx {

void server_note_push(tt_chan *c, uint64_t first, uint32_t n, int64_t arrival_ns) {
  TTServer *S = c->e->server;
  for (uint32_t i = 0; i < n; ++i) c->arrivals.emplace_back(first + i, arrival_ns);
  S->requests += n;
  int64_t prev = S->first_pending_ns.load(std::memory_order_relaxed);
  if (prev == 0 || arrival_ns < prev) S->first_pending_ns.store(arrival_ns, std::memory_order_relaxed);
}

void server_note_launch(tt_chan *c, uint64_t from, uint64_t to, uint64_t seq) {
  (void)from;
  TTServer *S = c->e->server;
  if (S->batches.empty() || S->batches.back().seq != seq) {
    S->batches.push_back({seq, {}, {}, nullptr});
    for (auto &ev : c->e->events)
      if (ev.first == seq) S->batches.back().done = ev.second;
  }
  auto &b = S->batches.back();
  b.chans.push_back(c);
  while (!c->arrivals.empty() && c->arrivals.front().first < to) {
    b.arrivals.push_back(c->arrivals.front().second);
    c->arrivals.pop_front();
  }
}

tt_status server_stamp_start(tt_engine *e, uint64_t seq, cudaStream_t st) {
  TTServer *S = e->server;
  cudaError_t err = tt_launch_stamp(S->d_stamp + TTServer::kRing + (seq % TTServer::kRing), st);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "start stamp: %s", cudaGetErrorString(err));
  ++e->launches;
  return TT_OK;
}

tt_status server_stamp(tt_engine *e, uint64_t seq, cudaStream_t st) {
  TTServer *S = e->server;
  cudaError_t err = tt_launch_stamp(S->d_stamp + (seq % TTServer::kRing), st);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "completion stamp: %s", cudaGetErrorString(err));
  ++e->launches;
  return TT_OK;
}

void server_count_wait(tt_engine *e, bool refused) {
  if (!e->server) return;
  if (refused) ++e->server->refused;
  else ++e->server->queued;
}

bool is_server_thread(const tt_engine *e) { return e->server && std::this_thread::get_id() == e->server->tid; }

int64_t server_queue_timeout_us(const tt_engine *e) {
  if (!e->server) return 0;
  const int32_t t = e->server->cfg.queue_timeout_us;
  return t == 0 ? 1000000 : (t < 0 ? 0 : t);
}

void admission_notify(tt_engine *e) {
  std::lock_guard<std::mutex> lk(e->admit_mu);
  e->admit_cv.notify_all();
}

}  // namespace ttx

namespace {

// Engine lock held: count every batch seen complete, release outputs if asked, wake waiting pushes.
void collect_completed(tt_engine *e) {
  TTServer *S = e->server;
  bool any = false;
  while (!S->batches.empty() && S->batches.front().seq <= e->completed_seq) {
    const TTServer::Batch &b = S->batches.front();
    const volatile unsigned long long *stamp = S->h_stamp + (b.seq % TTServer::kRing);
    const volatile unsigned long long *start = S->h_stamp + TTServer::kRing + (b.seq % TTServer::kRing);
    const int64_t t_done = (int64_t)*stamp - S->offset_ns;
    // device busy time: the union of the batches' spans (batches on different lanes overlap)
    const int64_t b0 = (int64_t)*start, b1 = (int64_t)*stamp;
    const int64_t from = std::max(b0, S->busy_until);
    if (b1 > from) S->gpu_ns += (double)(b1 - from);
    S->busy_until = std::max(S->busy_until, b1);
    if (!S->first_start || b0 < S->first_start) S->first_start = b0;
    S->last_end = std::max(S->last_end, b1);
    for (int64_t ta : b.arrivals) {
      if (ta < S->count_from_ns) continue;
      const double l = (double)(t_done - ta);
      S->lat_ns.push_back(l);
      if (l > S->deadline_ns) ++S->misses;
      ++S->completed;
    }
    ++S->n_batches;
    S->batched += b.arrivals.size();
    for (tt_chan *c : b.chans) {
      if (!c->e) continue;  // destroyed meanwhile
      ttx::update_chan(c);
      if (S->cfg.release_outputs && !c->cell) c->pulled_end = std::max(c->pulled_end, c->completed_end);
    }
    S->batches.pop_front();
    any = true;
  }
  // cells aggregated by completed batches free their ring slots too, also after a batch that only
  // aggregated (it carries no requests, so it is not in the list above)
  if (S->cfg.release_outputs)
    for (tt_cell *cl : e->cells) {
      while (!cl->inflight.empty() && cl->inflight.front().second <= e->completed_seq) {
        cl->completed_end = cl->inflight.front().first;
        cl->inflight.pop_front();
      }
      if (cl->completed_end > cl->pulled_end) {
        cl->pulled_end = cl->completed_end;
        any = true;
      }
    }
  if (any) e->room_cv.notify_all();
}

bool has_pending(const tt_engine *e) {
  for (const tt_chan *c : e->pending)
    if (c->has_trace && c->started && c->pushed_end > c->launched_end) return true;
  return false;
}

void server_loop(tt_engine *e) {
  TTServer *S = e->server;
  S->tid = std::this_thread::get_id();
  cudaSetDevice(e->device);
  const size_t max_inflight = S->cfg.max_inflight_batches ? S->cfg.max_inflight_batches : kDefaultInflight;
  for (;;) {
    bool launch = false, done = false;
    cudaEvent_t front = nullptr;
    {
      std::lock_guard<std::mutex> lk(e->mu);
      cudaError_t q = ttx::update_completed(e);
      if (q != cudaSuccess) {
        S->err = fail(TT_ERR_CUDA, "kernel failed: %s", cudaGetErrorString(q));
        S->err_msg = tt_last_error();
        break;
      }
      collect_completed(e);
      const bool pending = has_pending(e);
      if (!pending) S->first_pending_ns.store(0, std::memory_order_relaxed);  // launched meanwhile
      const size_t running = S->batches.size();
      const int64_t oldest = S->first_pending_ns.load(std::memory_order_relaxed);
      // a batch forms until its oldest request has waited the coalescing window: that bounds the
      // batch rate (each launch holds the engine lock for a few microseconds) and the wait.  An
      // uplink cell whose ring freed up aggregates at once even with no push pending: its members'
      // rings free only when it consumes their outputs, so waiting for a push could wait forever.
      const bool cell_work = !pending && !e->cells.empty() && ttx::cells_have_work(e);
      launch = running < max_inflight &&
               ((pending && oldest != 0 && now_ns() - oldest >= S->coalesce_ns) || cell_work);
      done = S->stop.load() && !pending && running == 0;
      if (!running && !pending && !done && !launch) {
        // idle: sleep until a push arrives (the pushes notify) or the stop flag
        std::unique_lock<std::mutex> ul(e->mu, std::adopt_lock);
        e->work_cv.wait_for(ul, std::chrono::microseconds(200));
        ul.release();
        continue;
      }
      if (running) front = S->batches.front().done;
    }
    if (!launch && !done && !front) {  // pending, nothing running: sleep out the window
      const int64_t oldest = S->first_pending_ns.load(std::memory_order_relaxed);
      const int64_t left = oldest ? S->coalesce_ns - (now_ns() - oldest) : 0;
      if (left > 2000) std::this_thread::sleep_for(std::chrono::nanoseconds(left - 1000));
      else std::this_thread::yield();
      continue;
    }
    if (done) break;
    if (launch) {
      S->first_pending_ns.store(0, std::memory_order_relaxed);
      const tt_status st = tt_engine_run(e);
      if (st != TT_OK) {
        S->err = st;
        S->err_msg = tt_last_error();
        break;
      }
      continue;
    }
    // a batch runs: poll its event without the engine lock until it completes or the pending
    // requests have gathered long enough for the next batch
    for (int spin = 0;; ++spin) {
      if (front && cudaEventQuery(front) != cudaErrorNotReady) break;
      const int64_t oldest = S->first_pending_ns.load(std::memory_order_relaxed);
      if (oldest != 0 && now_ns() - oldest >= S->coalesce_ns) break;
      if (S->stop.load() || spin > 4096) break;
      std::this_thread::yield();
    }
  }
  // after an error: wait for whatever was launched, so nothing the report counts is still running
  std::unique_lock<std::mutex> lk(e->mu);
  while (!S->batches.empty()) {
    if (ttx::update_completed(e) != cudaSuccess) break;
    collect_completed(e);
    lk.unlock();
    std::this_thread::yield();
    lk.lock();
  }
  e->room_cv.notify_all();
}

double percentile(const std::vector<double> &v, double p) {
  return v[std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5))];
}

}  // namespace

extern "C" {

tt_status tt_server_start(tt_engine *e, const tt_server_config *cfg) {
  if (!e || !cfg || cfg->struct_size < sizeof(tt_server_config)) return fail(TT_ERR_INVALID, "tt_server_start: bad argument");
  if (cfg->deadline_us < 0.0 || cfg->warmup_us < 0.0 || cfg->coalesce_us < 0.0)
    return fail(TT_ERR_INVALID, "tt_server_start: negative time");
  std::unique_ptr<TTServer> S(new TTServer);
  S->cfg = *cfg;
  S->deadline_ns = (cfg->deadline_us > 0.0 ? cfg->deadline_us : 500.0) * 1e3;
  if (cfg->coalesce_us > 0.0) S->coalesce_ns = (int64_t)(cfg->coalesce_us * 1e3);
  {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->server) return fail(TT_ERR_STATE, "a server already runs on this engine");
    if (cudaSetDevice(e->device) != cudaSuccess) return fail(TT_ERR_CUDA, "cudaSetDevice failed");
    if (cudaHostAlloc((void **)&S->h_stamp, sizeof(unsigned long long) * 2 * TTServer::kRing, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer((void **)&S->d_stamp, S->h_stamp, 0) != cudaSuccess) {
      if (S->h_stamp) cudaFreeHost(S->h_stamp);
      return fail(TT_ERR_CUDA, "stamp buffer: pinned mapped host memory unavailable");
    }
    std::memset(S->h_stamp, 0, sizeof(unsigned long long) * 2 * TTServer::kRing);
    // one launch lane per batch in flight: consecutive batches overlap on the GPU where the engine
    // allows it (no CUDA graphs, no cells)
    ttx::enable_lanes(e, cfg->max_inflight_batches ? (int)cfg->max_inflight_batches : kDefaultInflight);
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) {
      cudaFreeHost(S->h_stamp);
      return fail(TT_ERR_CUDA, "stream sync failed");
    }
    // device timer against the host steady clock: the shortest of 32 launch round trips
    int64_t best_rt = INT64_MAX;
    for (int i = 0; i < 32; ++i) {
      unsigned long long *slot = S->d_stamp + (TTServer::kRing - 1);
      const int64_t t0 = now_ns();
      cudaError_t err = tt_launch_stamp(slot, e->stream);
      if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
      const int64_t t1 = now_ns();
      if (err != cudaSuccess) {
        cudaFreeHost(S->h_stamp);
        return fail(TT_ERR_CUDA, "clock calibration: %s", cudaGetErrorString(err));
      }
      const int64_t dev = (int64_t)*(volatile unsigned long long *)(S->h_stamp + (TTServer::kRing - 1));
      if (t1 - t0 < best_rt) {
        best_rt = t1 - t0;
        S->offset_ns = dev - (t0 + (t1 - t0) / 2);
        S->calib_err_ns = (t1 - t0) / 2;
      }
    }
    S->count_from_ns = now_ns() + (int64_t)(cfg->warmup_us * 1e3);
    e->server = S.get();
  }
  TTServer *raw = S.release();
  raw->th = std::thread(server_loop, e);
  return TT_OK;
}

tt_status tt_server_stop(tt_engine *e, tt_server_report *out) {
  if (!e || (out && out->struct_size < sizeof(tt_server_report))) return fail(TT_ERR_INVALID, "tt_server_stop: bad argument");
  TTServer *S;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    S = e->server;
    if (!S) return fail(TT_ERR_STATE, "no server runs on this engine");
    S->stop.store(true);
    e->work_cv.notify_all();
  }
  S->th.join();
  tt_server_report r{};
  r.struct_size = sizeof r;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->server = nullptr;
    for (tt_chan *c : e->table)
      if (c) c->arrivals.clear();
    e->room_cv.notify_all();
  }
  r.requests = S->requests;
  r.completed = S->completed;
  r.queued = S->queued;
  r.refused = S->refused;
  r.batches = S->n_batches;
  r.deadline_misses = S->misses;
  r.mean_batch = S->n_batches ? (double)S->batched / (double)S->n_batches : 0.0;
  r.stamp_error_us = (double)S->calib_err_ns / 1e3;
  r.gpu_us_per_batch = S->n_batches ? S->gpu_ns / (double)S->n_batches / 1e3 : 0.0;
  r.gpu_busy = S->last_end > S->first_start ? S->gpu_ns / (double)(S->last_end - S->first_start) : 0.0;
  std::vector<double> &v = S->lat_ns;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    r.p50_us = percentile(v, 0.50) / 1e3;
    r.p99_us = percentile(v, 0.99) / 1e3;
    r.p999_us = percentile(v, 0.999) / 1e3;
    r.max_us = v.back() / 1e3;
    r.min_us = v.front() / 1e3;
    double sum = 0.0;
    for (double x : v) sum += x;
    r.mean_us = sum / (double)v.size() / 1e3;
  }
  const tt_status st = S->err;
  const std::string msg = S->err_msg;
  cudaFreeHost(S->h_stamp);
  delete S;
  if (out) *out = r;
  if (st != TT_OK) return fail(st, "server: %s", msg.c_str());
  return TT_OK;
}

tt_status tt_chan_create_queued(tt_engine *e, const tt_chan_config *cfg, int64_t timeout_us, tt_chan **out) {
  if (!e || !cfg || !out) return fail(TT_ERR_INVALID, "tt_chan_create_queued: bad argument");
  const int64_t deadline = timeout_us < 0 ? INT64_MAX : now_us() + timeout_us;
  std::unique_lock<std::mutex> lk(e->admit_mu);
  const uint64_t ticket = e->admit_next++;
  e->admit_queue.push_back(ticket);
  auto leave = [&]() {
    e->admit_queue.erase(std::find(e->admit_queue.begin(), e->admit_queue.end(), ticket));
    e->admit_cv.notify_all();
  };
  for (;;) {
    if (e->admit_queue.front() == ticket) {
      lk.unlock();
      const tt_status st = tt_chan_create(e, cfg, out);  // takes the engine lock
      const std::string msg = tt_last_error();
      lk.lock();
      if (st != TT_ERR_NO_MEMORY) {
        leave();
        if (st != TT_OK) return fail(st, "%s", msg.c_str());
        return TT_OK;
      }
    }
    const int64_t left = deadline - now_us();
    if (left <= 0) {
      leave();
      return fail(TT_ERR_NO_MEMORY, "admission: no room in the HBM budget within %lld us", (long long)timeout_us);
    }
    e->admit_cv.wait_for(lk, std::chrono::microseconds(std::min<int64_t>(left, 10000)));
  }
}

// ---------------------------------------------------------------- load generator
tt_status tt_engine_serve(tt_engine *e, const tt_serve_config *cfg, tt_serve_report *out) {
  if (!e || !cfg || !out || cfg->struct_size < sizeof(tt_serve_config))
    return fail(TT_ERR_INVALID, "tt_engine_serve: bad argument");
  if (!(cfg->duration_s > 0.0) || !(cfg->slot_period_us > 0.0) || cfg->warmup_s < 0.0 || cfg->jitter_us < 0.0)
    return fail(TT_ERR_INVALID, "tt_engine_serve: bad timing parameters");
  std::vector<tt_chan *> chans;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    for (tt_chan *c : e->table)
      if (c && c->has_trace) chans.push_back(c);
  }
  if (chans.empty()) return fail(TT_ERR_STATE, "tt_engine_serve: no channel with a trace");
  tt_server_config sc{};
  sc.struct_size = sizeof sc;
  sc.max_inflight_batches = cfg->max_inflight_batches;
  sc.release_outputs = cfg->release_outputs;
  sc.queue_timeout_us = -1;  // the generator queues its own arrivals instead of blocking
  sc.deadline_us = cfg->deadline_us;
  sc.warmup_us = cfg->warmup_s * 1e6;
  tt_status st = tt_server_start(e, &sc);
  if (st != TT_OK) return st;

  const int64_t period = (int64_t)(cfg->slot_period_us * 1e3), jitter = (int64_t)(cfg->jitter_us * 1e3);
  std::mt19937_64 rng(cfg->seed);
  std::exponential_distribution<double> expo(1.0 / (double)period);
  std::uniform_int_distribution<int64_t> jit(-jitter, jitter), phase(0, period);
  auto gap = [&]() -> int64_t { return std::max<int64_t>((int64_t)expo(rng) + jit(rng), 1000); };
  const int64_t t0 = now_ns();
  const int64_t t_warm = t0 + (int64_t)(cfg->warmup_s * 1e9), t_end = t_warm + (int64_t)(cfg->duration_s * 1e9);
  using Ev = std::pair<int64_t, uint32_t>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> heap;
  for (uint32_t u = 0; u < chans.size(); ++u) heap.push({t0 + phase(rng), u});
  // per-UE arrivals waiting for ring room (bounded): committed, with their own arrival times, as
  // soon as completed batches free the ring
  constexpr size_t kQueue = 64;
  std::vector<std::deque<int64_t>> waiting(chans.size());
  std::vector<uint32_t> waiting_ues;   // UEs whose queue is not empty
  std::vector<uint32_t> issued(chans.size(), 0);
  uint64_t requests = 0, refused = 0;
  size_t n_waiting = 0;
  // engine lock held: commit the UE's next slot with its own arrival time, if its ring has room
  auto commit = [&](uint32_t u, int64_t arrival) -> bool {
    tt_chan *c = chans[u];
    const uint64_t slot = c->started ? c->pushed_end : 0;
    if (ttx::check_room(c, slot, 1) != TT_OK) return false;
    ttx::mark_pushed_at(c, slot, 1, arrival);
    return true;
  };
  std::vector<Ev> due;
  for (;;) {
    const int64_t now = now_ns();
    due.clear();
    while (!heap.empty() && heap.top().first <= now && heap.top().first < t_end) {
      const Ev ev = heap.top();
      heap.pop();
      heap.push({ev.first + gap(), ev.second});
      if (cfg->max_slots_per_ue && issued[ev.second] >= cfg->max_slots_per_ue) continue;
      ++issued[ev.second];
      if (ev.first >= t_warm) ++requests;
      due.push_back(ev);
    }
    bool did = !due.empty();
    if (did || n_waiting) {  // one lock for the whole pass
      std::lock_guard<std::mutex> lk(e->mu);
      size_t k = 0;
      for (uint32_t u : waiting_ues) {
        while (!waiting[u].empty() && commit(u, waiting[u].front())) {
          waiting[u].pop_front();
          --n_waiting;
          did = true;
        }
        if (!waiting[u].empty()) waiting_ues[k++] = u;
      }
      waiting_ues.resize(k);
      for (const Ev &ev : due) {
        const uint32_t u = ev.second;
        if (waiting[u].empty() && commit(u, ev.first)) continue;
        if (waiting[u].size() < kQueue) {
          if (waiting[u].empty()) waiting_ues.push_back(u);
          waiting[u].push_back(ev.first);
          ++n_waiting;
        } else if (ev.first >= t_warm) {
          ++refused;  // the UE's queue is full: the engine is far behind this UE
        }
      }
      if (did) e->work_cv.notify_one();
    }
    if (now >= t_end && (n_waiting == 0 || now >= t_end + (int64_t)1e9)) break;
    if (!did) std::this_thread::yield();
  }
  tt_server_report r{};
  r.struct_size = sizeof r;
  st = tt_server_stop(e, &r);
  if (st != TT_OK) return st;
  tt_serve_report o{};
  o.requests = requests;
  o.refused = refused + (uint64_t)n_waiting;
  o.completed = r.completed;
  o.batches = r.batches;
  o.mean_batch = r.mean_batch;
  o.deadline_misses = r.deadline_misses;
  o.throughput = (double)r.completed / cfg->duration_s;
  o.p50_us = r.p50_us;
  o.p99_us = r.p99_us;
  o.p999_us = r.p999_us;
  o.max_us = r.max_us;
  o.mean_us = r.mean_us;
  o.stamp_error_us = r.stamp_error_us;
  o.gpu_us_per_batch = r.gpu_us_per_batch;
  o.gpu_busy = r.gpu_busy;
  *out = o;
  return TT_OK;
}

}  // extern "C"
