// Host side of the channel engine: the C ABI declared in include/tt_chan.h.
//
// One engine per GPU owns a CUDA stream, the device table of UE descriptors,
// and the admission budget.  One channel per UE link owns a slot ring for
// input and output on the device, its trace, and the cursors that keep its
// slots in order.  Per-UE isolation (paper Sec. III-C, "Parallelizing
// Convolution Computation") is kept by construction: every channel has its
// own ring, trace and descriptor, and no kernel mixes data of two UEs.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <deque>
#include <mutex>
#include <queue>
#include <random>
#include <unordered_map>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tt_chan.h"
#include "tt_engine_impl.h"
#include "tt_internal.h"

namespace ttx {

thread_local std::string g_err;

tt_status fail(tt_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

int64_t now_us() {
  return std::chrono::duration_cast<std::chrono::microseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

cudaError_t dev_alloc(tt_engine *e, void **p, size_t bytes) {
  *p = nullptr;
  if (!e->alloc_fn) return cudaMalloc(p, bytes);
  if (bytes == 0) return cudaSuccess;
  *p = e->alloc_fn(bytes, e->alloc_ctx);
  if (!*p) return cudaErrorMemoryAllocation;
  if (reinterpret_cast<uintptr_t>(*p) & 255) {  // the kernels' vector accesses rely on this
    e->free_fn(*p, e->alloc_ctx);
    *p = nullptr;
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

void dev_free(tt_engine *e, void *p) {
  if (!p) return;
  if (!e->alloc_fn) {
    cudaFree(p);
    return;
  }
  // the hook's memory may be reused as soon as it is returned: nothing of the engine may still use it
  if (e->quiesced) {
    e->free_fn(p, e->alloc_ctx);
    return;
  }
  sync_all(e);
  e->free_fn(p, e->alloc_ctx);
}

void sync_all(tt_engine *e) {
  for (cudaStream_t s : {e->stream, e->copy, e->h2d})
    if (s) cudaStreamSynchronize(s);
  for (int li = 0; li < e->n_lanes; ++li) {
    const TTLane &l = e->lanes[li];
    if (l.stream) cudaStreamSynchronize(l.stream);
    for (cudaStream_t s : l.side)
      if (s) cudaStreamSynchronize(s);
  }
  for (cudaStream_t s : e->side)
    if (s) cudaStreamSynchronize(s);
}

bool enable_lanes(tt_engine *e, int n) {
  n = std::min(n, tt_engine::kLanes);
  for (int li = e->n_lanes; li < n; ++li) {
    TTLane &l = e->lanes[li];
    cudaError_t err = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    for (int i = 0; i < tt_engine::kSide && err == cudaSuccess; ++i) {
      err = cudaStreamCreateWithFlags(&l.side[i], cudaStreamNonBlocking);
      if (err == cudaSuccess) err = cudaEventCreateWithFlags(&l.join[i], cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming);
    if (err == cudaSuccess) err = dmalloc(e, &l.d_segs, sizeof(TTSeg) * e->max_ues);
    if (err == cudaSuccess) err = dmalloc(e, &l.d_tcsegs, sizeof(TTSeg) * e->max_ues);
    if (err == cudaSuccess) err = dmalloc(e, &l.d_counters, sizeof(uint32_t) * e->counter_cap);
    if (err == cudaSuccess) err = dmalloc(e, &l.d_cursors, sizeof(unsigned long long) * e->max_ues);
    if (err == cudaSuccess) err = cudaMemsetAsync(l.d_counters, 0, sizeof(uint32_t) * e->counter_cap, l.stream);
    if (err != cudaSuccess) {  // stay on the lanes made so far
      dfree(e, l.d_segs);
      dfree(e, l.d_tcsegs);
      dfree(e, l.d_counters);
      dfree(e, l.d_cursors);
      for (int i = 0; i < tt_engine::kSide; ++i) {
        if (l.side[i]) cudaStreamDestroy(l.side[i]);
        if (l.join[i]) cudaEventDestroy(l.join[i]);
      }
      if (l.fork) cudaEventDestroy(l.fork);
      if (l.stream) cudaStreamDestroy(l.stream);
      l = TTLane{};
      cudaGetLastError();
      return e->n_lanes > 1;
    }
    e->n_lanes = li + 1;
  }
  return true;
}

NvtxScope::NvtxScope(const char *name) { nvtxRangePushA(name); }
NvtxScope::~NvtxScope() { nvtxRangePop(); }

}  // namespace ttx

using ttx::dfree;
using ttx::dmalloc;

using ttx::fail;
using ttx::now_ns;
using ttx::now_us;

namespace {

cudaEvent_t get_event(tt_engine *e) {
  if (!e->pool.empty()) {
    cudaEvent_t ev = e->pool.back();
    e->pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return ev;
}

// Poll batch events in order; returns the first hard CUDA error seen.
cudaError_t update_completed(tt_engine *e) {
  while (!e->events.empty()) {
    cudaError_t q = cudaEventQuery(e->events.front().second);
    if (q == cudaErrorNotReady) break;
    if (q != cudaSuccess) return q;
    e->completed_seq = e->events.front().first;
    e->pool.push_back(e->events.front().second);
    e->events.pop_front();
  }
  return cudaSuccess;
}

void update_chan(tt_chan *c) {
  while (!c->inflight.empty() && c->inflight.front().second <= c->e->completed_seq) {
    c->completed_end = c->inflight.front().first;
    c->inflight.pop_front();
  }
}

cudaEvent_t event_of(tt_engine *e, uint64_t seq) {
  for (auto &p : e->events)
    if (p.first == seq) return p.second;
  return nullptr;
}

// Wait (bounded) until batch `seq` is complete.
tt_status wait_seq(tt_engine *e, uint64_t seq, int64_t timeout_us, std::unique_lock<std::mutex> &lk) {
  const int64_t deadline = timeout_us < 0 ? INT64_MAX : now_us() + timeout_us;
  for (;;) {
    cudaError_t q = update_completed(e);
    if (q != cudaSuccess) return fail(TT_ERR_CUDA, "kernel failed: %s", cudaGetErrorString(q));
    if (e->completed_seq >= seq) return TT_OK;
    if (timeout_us == 0) return fail(TT_ERR_TIMEOUT, "slot still running");
    if (timeout_us < 0) {
      cudaEvent_t ev = event_of(e, seq);
      if (ev) {
        lk.unlock();
        cudaError_t s = cudaEventSynchronize(ev);
        lk.lock();
        if (s != cudaSuccess) return fail(TT_ERR_CUDA, "kernel failed: %s", cudaGetErrorString(s));
      }
      continue;
    }
    if (now_us() > deadline) return fail(TT_ERR_TIMEOUT, "slot still running after %lld us",
                                         (long long)timeout_us);
    lk.unlock();
    std::this_thread::yield();
    lk.lock();
  }
}

int pick_dclass(int d_max) {
  if (d_max <= TT_DCLASS0) return 0;
  if (d_max <= TT_DCLASS1) return 1;
  if (d_max <= TT_DCLASS2) return 2;
  return 3;
}

// Work-item geometry of a channel for samples-per-thread spt and tpb threads per CTA: (chunk
// table, largest symbols touched).
std::vector<int32_t> chunk_table(const std::vector<uint32_t> &L, int spt, int tpb, int *max_touched) {
  int n = 0;
  for (uint32_t v : L) n += (int)v;
  const int items = (n / spt + tpb - 1) / tpb;
  std::vector<int32_t> L32(L.begin(), L.end()), chunks(items);
  tt_conv_chunk_info(spt, tpb, L32.data(), (int)L32.size(), chunks.data(), items);
  *max_touched = 1;
  for (int32_t v : chunks) *max_touched = std::max(*max_touched, (int)(v >> 16));
  return chunks;
}

// Candidate samples-per-thread values of a channel, largest first: each divides every
// symbol length; 16 only with at most 2 Rx antennas; none above the engine's cap.
std::vector<int> spt_candidates(const std::vector<uint32_t> &L, uint32_t cap, uint32_t n_rx, uint32_t n_tx) {
  std::vector<int> out;
  // Default cap 8: small batches (the serving loop) keep more, shorter work items in flight.  Bulk
  // runs of single-antenna channels go faster at 16 (4.58 ms against 4.72 ms for 16,000 40 MHz,
  // 24-tap UE-slots); the engine's samples_per_thread setting asks for it.
  (void)n_tx;
  if (cap == 0) cap = 8;
  for (int s : {16, 8, 4, 2, 1}) {
    if ((uint32_t)s > cap) continue;
    if (s == 16 && n_rx > 2) continue;
    bool ok = true;
    for (uint32_t v : L) ok = ok && (v % (uint32_t)s == 0);
    if (ok) out.push_back(s);
  }
  return out;
}

// Copy [first, first+n) slots between a linear buffer and the ring (<= 2 copies).
cudaError_t ring_copy(int16_t *ring, size_t slot_elems, int Q, uint64_t first, uint32_t n, const void *src,
                      void *dst, cudaMemcpyKind kind, cudaStream_t st, bool to_ring) {
  uint32_t done = 0;
  while (done < n) {
    const uint32_t pos = (uint32_t)((first + done) % (uint64_t)Q);
    const uint32_t run = std::min<uint32_t>(n - done, (uint32_t)Q - pos);
    const size_t bytes = (size_t)run * slot_elems * sizeof(int16_t);
    int16_t *r = ring + (size_t)pos * slot_elems;
    cudaError_t err;
    if (to_ring)
      err = cudaMemcpyAsync(r, static_cast<const int16_t *>(src) + (size_t)done * slot_elems, bytes, kind, st);
    else
      err = cudaMemcpyAsync(static_cast<int16_t *>(dst) + (size_t)done * slot_elems, r, bytes, kind, st);
    if (err != cudaSuccess) return err;
    done += run;
  }
  return cudaSuccess;
}

tt_status upload_desc(tt_chan *c) {
  tt_engine *e = c->e;
  TT_CK(cudaMemcpyAsync(e->d_ues + c->index, &c->desc, sizeof(TTUEDesc), cudaMemcpyHostToDevice, e->stream));
  // the host copy of the descriptor may change again before the copy runs
  TT_CK(cudaStreamSynchronize(e->stream));
  return TT_OK;
}

tt_status check_room(tt_chan *c, uint64_t first, uint32_t n) {
  const uint64_t start = c->started ? c->pulled_end : first;
  if (c->started && first != c->pushed_end)
    return fail(TT_ERR_STATE, "slot %llu pushed, expected %llu", (unsigned long long)first,
                (unsigned long long)c->pushed_end);
  if (first + n - start + (uint64_t)c->hist > (uint64_t)c->Q)
    return fail(TT_ERR_AGAIN, "slot ring full (depth %d): pull or release outputs first", c->Q);
  return TT_OK;
}

void mark_pushed_at(tt_chan *c, uint64_t first, uint32_t n, int64_t arrival_ns) {
  if (!c->started) {
    c->started = true;
    c->start_slot = first;
    c->pushed_end = c->launched_end = c->completed_end = c->pulled_end = first;
  }
  c->pushed_end = first + n;
  if (!c->in_pending) {
    c->in_pending = true;
    c->e->pending.push_back(c);
  }
  if (c->e->server) ttx::server_note_push(c, first, n, arrival_ns);
}

void mark_pushed(tt_chan *c, uint64_t first, uint32_t n) { mark_pushed_at(c, first, n, now_ns()); }

bool valid_chan(const tt_chan *c) { return c && c->e; }

// Switch a channel's tiled-kernel geometry to spt samples per thread and tpb threads per CTA
// (engine lock held).
tt_status set_geom(tt_chan *c, int spt, int tpb) {
  int touched = 1;
  std::vector<int32_t> chunks = chunk_table(c->sym_len, spt, tpb, &touched);
  int32_t *d_chunks = nullptr;
  cudaError_t err = dmalloc(c->e, &d_chunks, chunks.size() * sizeof(int32_t));
  if (err == cudaSuccess)
    err = cudaMemcpy(d_chunks, chunks.data(), chunks.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
  // streams are not ordered after the default stream: let them land before any kernel reads them
  if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
  if (err != cudaSuccess) {
    dfree(c->e, d_chunks);
    return fail(TT_ERR_CUDA, "chunk table: %s", cudaGetErrorString(err));
  }
  dfree(c->e, c->d_chunks);
  c->d_chunks = d_chunks;
  c->spt = spt;
  c->tpb = tpb;
  c->max_sym_touched = touched;
  TTUEDesc &d = c->desc;
  d.chunk_info = d_chunks;
  d.spt = spt;
  d.tpb = tpb;
  d.groups = c->n / spt;
  d.items_per_slot = (int)chunks.size();
  int b = 0, g = 0;
  for (int j = 0; j < d.nsym; ++j) {
    d.sym_start[j] = b;
    d.grp_start[j] = g;
    b += (int)c->sym_len[j];
    g += (int)c->sym_len[j] / spt;
  }
  d.sym_start[d.nsym] = b;
  d.grp_start[d.nsym] = g;
  d.dpad = (d.d_max + spt - 1) / spt * spt;
  return TT_OK;
}

// Sparse convolution is active when top_n keeps fewer taps than the trace has.
bool sparse(const tt_chan *c) { return c->desc.top_n > 0 && c->desc.top_n < c->desc.n_taps; }

// Length of the kernel's per-item delay-offset array: the trace's taps, or with sparse convolution
// the compacted lists of every touched symbol and link (at most tap_need entries).
int k_need(const tt_chan *c, int tap_need) { return sparse(c) ? std::max(c->desc.n_taps, tap_need) : c->desc.n_taps; }

// Shared-memory need of a traced channel at spt samples per thread and tpb threads per CTA (0 if
// it does not fit); with sparse convolution the delay-offset array holds the compacted lists of
// every touched symbol.
size_t smem_need(const tt_chan *c, int spt, int tpb, int *tap_need) {
  int touched = 1;
  chunk_table(c->sym_len, spt, tpb, &touched);
  *tap_need = touched * (int)(c->cfg.n_rx * c->cfg.n_tx * (uint32_t)c->desc.n_taps);
  const size_t b = tt_conv_smem_bytes(spt, tpb, c->dclass, (int)c->cfg.n_tx, *tap_need, k_need(c, *tap_need));
  return b <= 200 * 1024 ? b : 0;
}

// Switch a traced channel to (spt, tpb) and refresh its launch parameters (engine lock held).
tt_status apply_geom(tt_chan *c, int spt, int tpb) {
  int need = 0;
  const size_t b = smem_need(c, spt, tpb, &need);
  if (!b) return fail(TT_ERR_INVALID, "%d samples per thread at %d threads does not fit", spt, tpb);
  tt_status st = set_geom(c, spt, tpb);
  if (st != TT_OK) return st;
  c->tap_need = need;
  c->smem = b;
  return TT_OK;
}

// ---- batched launch planning (engine lock held) ----
struct PlanGroup {
  size_t seg0 = 0;
  int nseg = 0;
  uint32_t items = 0;
  size_t smem = 0;
  int spt = 1, tpb = TT_TPB, nrx = 1, ntx = 1, dclass = 0, tap_max = 1, k_max = 1, grid = 1;
  int topn = 0;  // the group's UEs use sparse convolution
};
struct Plan {
  std::vector<TTSeg> segs;
  std::vector<PlanGroup> groups;
  std::vector<tt_chan *> chans;  // in segment order
  std::vector<uint64_t> key;     // shape: (UE, slots, variant) per segment
};

// One segment per channel (slots [first[i], first[i] + count[i])), grouped by kernel variant,
// heaviest channels first inside a group; grid sizes from the occupancy of each variant.
tt_status build_plan(tt_engine *e, const std::vector<tt_chan *> &chans, const std::vector<uint64_t> &first,
                     const std::vector<uint64_t> &count, Plan &p) {
  std::vector<size_t> order(chans.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  auto vkey = [&](size_t i) {
    const tt_chan *c = chans[i];
    return ((((c->spt * 8 + (int)c->cfg.n_rx) * 8 + (int)c->cfg.n_tx) * 8 + c->dclass) * 2 + (sparse(c) ? 1 : 0)) * 2 +
           (c->tpb == TT_TPB_WIDE ? 1 : 0);
  };
  auto cost = [&](size_t i) {
    const tt_chan *c = chans[i];
    return (double)c->desc.n_taps * c->cfg.n_tx * c->cfg.n_rx;
  };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    if (vkey(a) != vkey(b)) return vkey(a) < vkey(b);
    return cost(a) > cost(b);
  });
  int cur_key = -1;
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const size_t i = order[oi];
    tt_chan *c = chans[i];
    if (count[i] == 0) continue;
    if (p.groups.empty() || vkey(i) != cur_key) {
      cur_key = vkey(i);
      PlanGroup g;
      g.seg0 = p.segs.size();
      g.spt = c->spt;
      g.tpb = c->tpb;
      g.nrx = (int)c->cfg.n_rx;
      g.ntx = (int)c->cfg.n_tx;
      g.dclass = c->dclass;
      g.topn = sparse(c) ? 1 : 0;
      p.groups.push_back(g);
    }
    PlanGroup &g = p.groups.back();
    TTSeg sg{};
    sg.first_slot = first[i];
    sg.ue = c->index;
    sg.n_slots = (uint32_t)count[i];
    sg.item_begin = g.items;
    sg.items = sg.n_slots * (uint32_t)c->desc.items_per_slot;
    g.items += sg.items;
    g.tap_max = std::max(g.tap_max, c->tap_need);
    g.k_max = std::max(g.k_max, k_need(c, c->tap_need));
    ++g.nseg;
    p.segs.push_back(sg);
    p.chans.push_back(c);
    p.key.push_back(((uint64_t)c->index << 40) ^ ((uint64_t)count[i] << 8) ^ (uint64_t)vkey(i));
  }
  if ((int)p.groups.size() > e->counter_cap) return fail(TT_ERR_INVALID, "too many kernel variants in one run");
  for (PlanGroup &g : p.groups) {
    g.smem = tt_conv_smem_bytes(g.spt, g.tpb, g.dclass, g.ntx, g.tap_max, g.k_max);
    TTLaunch L{};
    L.spt = g.spt;
    L.tpb = g.tpb;
    L.nrx = g.nrx;
    L.ntx = g.ntx;
    L.dclass = g.dclass;
    L.topn = g.topn;
    L.smem = g.smem;
    L.grid = -1;  // occupancy query
    cudaError_t err = tt_launch_conv_fp32(L, e->stream);
    if (err != cudaSuccess) return fail(TT_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(err));
    g.grid = (int)std::min<uint64_t>((uint64_t)(-L.grid) * e->num_sms, g.items);
  }
  return TT_OK;
}

cudaError_t enqueue_plan(tt_engine *e, const Plan &p, const TTSeg *d_segs, const unsigned long long *cursors,
                         TTLane &ln) {
  if (e->persistent) {
    cudaError_t err = cudaMemsetAsync(ln.d_counters, 0, sizeof(uint32_t) * p.groups.size(), ln.stream);
    if (err != cudaSuccess) return err;
  }
  // largest variant on the engine stream, the others on side branches that start with it
  std::vector<size_t> order(p.groups.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return (double)p.groups[a].items * p.groups[a].k_max * p.groups[a].nrx * p.groups[a].spt >
           (double)p.groups[b].items * p.groups[b].k_max * p.groups[b].nrx * p.groups[b].spt;
  });
  const int n_side = (int)std::min<size_t>(order.size() > 0 ? order.size() - 1 : 0, tt_engine::kSide);
  if (n_side > 0) {
    cudaError_t err = cudaEventRecord(ln.fork, ln.stream);
    for (int i = 0; i < n_side && err == cudaSuccess; ++i) err = cudaStreamWaitEvent(ln.side[i], ln.fork, 0);
    if (err != cudaSuccess) return err;
  }
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const size_t gi = order[oi];
    const PlanGroup &g = p.groups[gi];
    TTLaunch L{};
    L.ues = e->d_ues;
    L.segs = d_segs + g.seg0;
    L.n_segs = g.nseg;
    L.total_items = g.items;
    L.counter = e->persistent ? ln.d_counters + gi : nullptr;
    L.spt = g.spt;
    L.tpb = g.tpb;
    L.nrx = g.nrx;
    L.ntx = g.ntx;
    L.dclass = g.dclass;
    L.tap_max = g.tap_max;
    L.k_max = g.k_max;
    L.topn = g.topn;
    L.smem = g.smem;
    L.grid = g.grid;
    L.cursors = cursors;
    L.check.report = e->d_check;
    L.check.shrink = e->check_shrink;
    cudaStream_t st = oi == 0 || n_side == 0 ? ln.stream : ln.side[(oi - 1) % n_side];
    cudaError_t err = tt_launch_conv_fp32(L, st);
    if (err != cudaSuccess) return err;
  }
  for (int i = 0; i < n_side; ++i) {
    cudaError_t err = cudaEventRecord(ln.join[i], ln.side[i]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(ln.stream, ln.join[i], 0);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Direct launch: the work list is uploaded from the host and the device cursors are not used.
tt_status launch_direct(tt_engine *e, const Plan &p, TTLane &ln) {
  // every lane's list holds max_ues segments (one per channel), sized when the engine or lane was made
  if (p.segs.size() > e->seg_cap) return fail(TT_ERR_STATE, "work list of %zu segments", p.segs.size());
  TT_CK(cudaMemcpyAsync(ln.d_segs, p.segs.data(), sizeof(TTSeg) * p.segs.size(), cudaMemcpyHostToDevice,
                        ln.stream));
  cudaError_t err = enqueue_plan(e, p, ln.d_segs, nullptr, ln);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "tiled launch: %s", cudaGetErrorString(err));
  e->launches += p.groups.size();
  for (tt_chan *c : p.chans)
    for (uint64_t &v : c->dev_cursor) v = UINT64_MAX;  // the device cursors did not follow
  return TT_OK;
}

tt_status launch_cached_graph(tt_engine *e, const std::vector<tt_chan *> &chans, const std::vector<TTSeg> &segs,
                              int li);

// Forget the cached graph (channel set or geometry changed).  Engine lock held.
void drop_graph(tt_engine *e) {
  bool any = false;
  for (int li = 0; li < e->n_lanes; ++li) any = any || e->lanes[li].gexec;
  if (any) {
    ttx::sync_all(e);
    for (int li = 0; li < e->n_lanes; ++li)
      if (e->lanes[li].gexec) {
        cudaGraphExecDestroy(e->lanes[li].gexec);
        e->lanes[li].gexec = nullptr;
      }
  }
  e->gkey.clear();
  e->gchans.clear();
  e->gcounts.clear();
  e->gplan_chans.clear();
}

// Lanes a run's batch may use: while a server runs or graphs are replayed, and without cells.
int rotation(const tt_engine *e) {
  return (e->n_lanes > 1 && e->cells.empty() && (e->server || e->graphs)) ? e->n_lanes : 1;
}

// Graph launch: a run of the same shape as the cached graph replays it; the slot each run
// starts at comes from the device cursors, which the graph's last node advances.  Each lane of
// the rotation has its own instance (its counters, streams and cursors), built together.
tt_status launch_graph(tt_engine *e, const Plan &p, int li) {
  const int stride = rotation(e);
  if (e->gkey.empty() || p.key != e->gkey || stride != e->gstride || !e->lanes[li].gexec) {
    drop_graph(e);  // waits for every lane: old instances may still read d_gsegs
    if (p.segs.size() > e->gseg_cap) {
      dfree(e, e->d_gsegs);
      e->d_gsegs = nullptr;
      e->gseg_cap = 0;
      TT_CK(dmalloc(e, &e->d_gsegs, sizeof(TTSeg) * p.segs.size() * 2));
      e->gseg_cap = p.segs.size() * 2;
    }
    TT_CK(cudaMemcpy(e->d_gsegs, p.segs.data(), sizeof(TTSeg) * p.segs.size(), cudaMemcpyHostToDevice));
    // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
    // streams are not ordered after the default stream: let them land before any kernel reads them
    TT_CK(cudaStreamSynchronize(nullptr));
    for (int l = 0; l < stride; ++l) {
      TTLane &ln = e->lanes[l];
      cudaGraph_t graph = nullptr;
      TT_CK(cudaStreamBeginCapture(ln.stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t err = enqueue_plan(e, p, e->d_gsegs, ln.d_cursors, ln);
      if (err == cudaSuccess)
        err = tt_launch_advance(e->d_gsegs, (int)p.segs.size(), ln.d_cursors, (unsigned)stride, ln.stream);
      cudaError_t err2 = cudaStreamEndCapture(ln.stream, &graph);
      if (err == cudaSuccess) err = err2;
      if (err == cudaSuccess) err = cudaGraphInstantiate(&ln.gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (err != cudaSuccess) {
        ln.gexec = nullptr;
        drop_graph(e);
        return fail(TT_ERR_CUDA, "graph build: %s", cudaGetErrorString(err));
      }
    }
    for (tt_chan *c : p.chans)
      for (uint64_t &v : c->dev_cursor) v = UINT64_MAX;  // fresh instances: every cursor is set on first use
    e->gkey = p.key;
    e->gstride = stride;
    e->graph_nodes = p.groups.size();
    e->gsegs_host = p.segs;
    ++e->graph_builds;
  }
  return launch_cached_graph(e, p.chans, p.segs, li);
}

// Replay lane li's instance of the cached graph for channels `chans` (segment order) starting at
// the given slots.
tt_status launch_cached_graph(tt_engine *e, const std::vector<tt_chan *> &chans, const std::vector<TTSeg> &segs,
                              int li) {
  TTLane &ln = e->lanes[li];
  // bring this lane's stale device cursors in line with the host's view
  std::vector<unsigned long long> fix(chans.size());
  bool any = false;
  for (size_t i = 0; i < chans.size(); ++i) {
    tt_chan *c = chans[i];
    if (c->dev_cursor[li] != segs[i].first_slot) {
      fix[i] = segs[i].first_slot;
      TT_CK(cudaMemcpyAsync(ln.d_cursors + c->index, &fix[i], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            ln.stream));
      any = true;
    }
  }
  if (any) TT_CK(cudaStreamSynchronize(ln.stream));  // fix[] lives on this stack frame
  TT_CK(cudaGraphLaunch(ln.gexec, ln.stream));
  ++e->graph_launches;
  e->launches += e->graph_nodes;
  for (size_t i = 0; i < chans.size(); ++i)
    chans[i]->dev_cursor[li] = segs[i].first_slot + (uint64_t)e->gstride * segs[i].n_slots;
  return TT_OK;
}

// Tensor-core channels: one item per (UE, slot, symbol), BF16 and FP16 channels in separate launches.
tt_status launch_tc(tt_engine *e, const std::vector<tt_chan *> &chans, TTLane &ln) {
  {  // failure-detection tests: the kernel issues no MMA, so its bounded waits run out
    const char *v = std::getenv("TT_TEST_TC_NO_MMA");
    e->tc_no_mma = (v && v[0] == '1') ? 1 : 0;
  }
  std::vector<TTSeg> segs;
  int n16 = 0;
  for (int pass = 0; pass < 2; ++pass)  // BF16 channels first, then FP16
    for (tt_chan *c : chans) {
      const bool fp16 = c->cfg.precision == TT_FP16_TC;
      if ((int)fp16 != pass) continue;
      TTSeg sg{};
      sg.first_slot = c->launched_end;
      sg.ue = c->index;
      sg.n_slots = (uint32_t)(c->pushed_end - c->launched_end);
      sg.items = sg.n_slots * (uint32_t)c->desc.items_per_slot;
      segs.push_back(sg);
      n16 += fp16;
    }
  if (segs.size() > e->tcseg_cap) return fail(TT_ERR_STATE, "tensor-core work list of %zu segments", segs.size());
  const size_t nbf = segs.size() - (size_t)n16;
  uint32_t acc = 0;
  for (size_t i = 0; i < segs.size(); ++i) {
    if (i == nbf) acc = 0;  // item numbering restarts for the FP16 launch
    segs[i].item_begin = acc;
    acc += segs[i].items;
  }
  TT_CK(cudaMemcpyAsync(ln.d_tcsegs, segs.data(), sizeof(TTSeg) * segs.size(), cudaMemcpyHostToDevice,
                        ln.stream));
  for (int pass = 0; pass < 2; ++pass) {
    const size_t s0 = pass ? nbf : 0, s1 = pass ? segs.size() : nbf;
    if (s0 == s1) continue;
    uint32_t items = 0;
    for (size_t i = s0; i < s1; ++i) items += segs[i].items;
    TTLaunch L{};
    L.ues = e->d_ues;
    L.segs = ln.d_tcsegs + s0;
    L.n_segs = (int)(s1 - s0);
    L.total_items = items;
    L.counter = nullptr;
    L.check.report = e->d_check;
    L.check.shrink = e->check_shrink;
    L.grid = -1;
    cudaError_t err = tt_launch_toeplitz_tc(L, pass == 1, e->d_status, e->tc_no_mma, ln.stream);
    if (err != cudaSuccess) return fail(TT_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(err));
    L.grid = (int)std::min<uint64_t>((uint64_t)(-L.grid) * e->num_sms, items);
    err = tt_launch_toeplitz_tc(L, pass == 1, e->d_status, e->tc_no_mma, ln.stream);
    if (err != cudaSuccess) return fail(TT_ERR_CUDA, "tensor-core launch: %s", cudaGetErrorString(err));
    ++e->launches;
  }
  return TT_OK;
}

}  // namespace

namespace ttx {
cudaEvent_t get_event(tt_engine *e) { return ::get_event(e); }
std::vector<int> spt_candidates(const std::vector<uint32_t> &L, uint32_t cap, uint32_t n_rx, uint32_t n_tx) {
  return ::spt_candidates(L, cap, n_rx, n_tx);
}
size_t smem_need(const tt_chan *c, int spt, int tpb, int *tap_need) { return ::smem_need(c, spt, tpb, tap_need); }
tt_status apply_geom(tt_chan *c, int spt, int tpb) { return ::apply_geom(c, spt, tpb); }
tt_status upload_desc(tt_chan *c) { return ::upload_desc(c); }
void drop_graph(tt_engine *e) { ::drop_graph(e); }
tt_status time_batch(tt_engine *e, const std::vector<tt_chan *> &chans, const std::vector<uint64_t> &first,
                     const std::vector<uint64_t> &count, int reps, cudaEvent_t a, cudaEvent_t b, float *best_ms) {
  Plan plan;
  tt_status st = build_plan(e, chans, first, count, plan);
  if (st != TT_OK) return st;
  if ((st = launch_direct(e, plan, e->lanes[0])) != TT_OK) return st;  // warm-up
  *best_ms = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, e->stream);
    if ((st = launch_direct(e, plan, e->lanes[0])) != TT_OK) return st;
    cudaEventRecord(b, e->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) return fail(TT_ERR_CUDA, "autotune: timing failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *best_ms = std::min(*best_ms, ms);
  }
  return TT_OK;
}
cudaError_t update_completed(tt_engine *e) { return ::update_completed(e); }
void update_chan(tt_chan *c) { ::update_chan(c); }
tt_status check_room(tt_chan *c, uint64_t first, uint32_t n) { return ::check_room(c, first, n); }
void mark_pushed(tt_chan *c, uint64_t first, uint32_t n) { ::mark_pushed(c, first, n); }
void mark_pushed_at(tt_chan *c, uint64_t first, uint32_t n, int64_t arrival_ns) {
  ::mark_pushed_at(c, first, n, arrival_ns);
}
tt_status wait_seq(tt_engine *e, uint64_t seq, int64_t timeout_us, std::unique_lock<std::mutex> &lk) {
  return ::wait_seq(e, seq, timeout_us, lk);
}
std::vector<int32_t> chunk_table(const std::vector<uint32_t> &L, int spt, int tpb, int *max_touched) {
  return ::chunk_table(L, spt, tpb, max_touched);
}
int pick_dclass(int d_max) { return ::pick_dclass(d_max); }
tt_status set_geom(tt_chan *c, int spt, int tpb) { return ::set_geom(c, spt, tpb); }
bool sparse(const tt_chan *c) { return ::sparse(c); }
bool valid_chan(const tt_chan *c) { return ::valid_chan(c); }
cudaError_t ring_copy(int16_t *ring, size_t slot_elems, int Q, uint64_t first, uint32_t n, const void *src, void *dst,
                      cudaMemcpyKind kind, cudaStream_t st, bool to_ring) {
  return ::ring_copy(ring, slot_elems, Q, first, n, src, dst, kind, st, to_ring);
}
}  // namespace ttx

int32_t tt_set_error(int32_t status, const char *msg) {
  ttx::g_err = msg ? msg : "";
  return status;
}

// =========================================================================
extern "C" {

const char *tt_last_error(void) { return ttx::g_err.c_str(); }
int32_t tt_abi_version(void) { return TT_CHAN_ABI_VERSION; }

tt_status tt_engine_create(const tt_engine_config *cfg, tt_engine **out) {
  if (!cfg || !out || cfg->struct_size < sizeof(tt_engine_config))
    return fail(TT_ERR_INVALID, "tt_engine_create: bad config");
  if (cfg->form > TT_FORM_PLAIN) return fail(TT_ERR_INVALID, "unknown form %u", cfg->form);
  if (cfg->samples_per_thread && cfg->samples_per_thread != 1 && cfg->samples_per_thread != 2 &&
      cfg->samples_per_thread != 4 && cfg->samples_per_thread != 8 && cfg->samples_per_thread != 16)
    return fail(TT_ERR_INVALID, "samples_per_thread must be 0, 1, 2, 4, 8 or 16");
  if (cfg->threads_per_block && cfg->threads_per_block != TT_TPB && cfg->threads_per_block != TT_TPB_WIDE)
    return fail(TT_ERR_INVALID, "threads_per_block must be 0, %d or %d", TT_TPB, TT_TPB_WIDE);
  int ndev = 0;
  cudaError_t q = cudaGetDeviceCount(&ndev);
  if (q != cudaSuccess || ndev == 0) return fail(TT_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(q));
  if (cfg->device < 0 || cfg->device >= ndev) return fail(TT_ERR_CUDA, "no CUDA device %d", cfg->device);
  TT_CK(cudaSetDevice(cfg->device));
  tt_engine *e = new tt_engine();
  e->device = cfg->device;
  e->budget = cfg->hbm_budget_bytes;
  e->form = cfg->form;
  e->max_ues = cfg->max_ues ? cfg->max_ues : 1024;
  e->spt_override = cfg->samples_per_thread;
  e->tpb_override = cfg->threads_per_block;
  e->persistent = cfg->persistent;
  e->graphs = cfg->struct_size >= offsetof(tt_engine_config, graphs) + sizeof(uint32_t) && cfg->graphs != 0;
  if (cfg->struct_size >= offsetof(tt_engine_config, alloc_ctx) + sizeof(void *)) {
    if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr)) {
      delete e;
      return fail(TT_ERR_INVALID, "dev_alloc and dev_free must be set together");
    }
    e->alloc_fn = cfg->dev_alloc;
    e->free_fn = cfg->dev_free;
    e->alloc_ctx = cfg->alloc_ctx;
  }
  cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
  ttx::tune_load(e);  // choices stored for this device model (TT_TUNE_CACHE)
  e->table.assign(e->max_ues, nullptr);
  cudaError_t err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->copy, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->h2d, cudaStreamNonBlocking);
  for (int i = 0; i < tt_engine::kSide && err == cudaSuccess; ++i) {
    err = cudaStreamCreateWithFlags(&e->side[i], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->join[i], cudaEventDisableTiming);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_ues, sizeof(TTUEDesc) * e->max_ues);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_counters, sizeof(uint32_t) * e->counter_cap);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_cursors, sizeof(unsigned long long) * e->max_ues);
  // work lists hold at most one run of slots per channel: sized once, never regrown during runs
  if (err == cudaSuccess) err = dmalloc(e, &e->d_segs, sizeof(TTSeg) * e->max_ues);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_gsegs, sizeof(TTSeg) * e->max_ues);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_tcsegs, sizeof(TTSeg) * e->max_ues);
  if (err == cudaSuccess) e->seg_cap = e->gseg_cap = e->tcseg_cap = e->max_ues;
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->lane_pre, cudaEventDisableTiming);
  if (err == cudaSuccess) {  // lane 0 is the engine's own stream and lists
    TTLane &l0 = e->lanes[0];
    l0.stream = e->stream;
    for (int i = 0; i < tt_engine::kSide; ++i) {
      l0.side[i] = e->side[i];
      l0.join[i] = e->join[i];
    }
    l0.fork = e->fork;
    l0.d_segs = e->d_segs;
    l0.d_tcsegs = e->d_tcsegs;
    l0.d_counters = e->d_counters;
    l0.d_cursors = e->d_cursors;
  }
  // graph replays overlap consecutive steps on four lanes (about 10% less GPU time per step of
  // 256 mixed UEs than one stream; eight measured the same within noise); an engine that cannot
  // make them stays on one
  if (err == cudaSuccess && e->graphs) ttx::enable_lanes(e, 4);
  if (err == cudaSuccess) err = dmalloc(e, &e->d_status, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(e->d_status, 0, sizeof(int));
  if (err == cudaSuccess) err = dmalloc(e, &e->d_check, 2 * sizeof(uint32_t));
  if (err == cudaSuccess) err = cudaMemset(e->d_check, 0, 2 * sizeof(uint32_t));
  // a device memset may return before it lands, and the engine's non-blocking streams are not
  // ordered after the default stream: finish it before any kernel can write these words
  if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
  if (err != cudaSuccess) {
    tt_engine_destroy(e);
    return fail(TT_ERR_CUDA, "engine setup: %s", cudaGetErrorString(err));
  }
  *out = e;
  return TT_OK;
}

tt_status tt_engine_destroy(tt_engine *e) {
  if (!e) return fail(TT_ERR_INVALID, "null engine");
  if (e->server) tt_server_stop(e, nullptr);  // its thread launches on this engine
  cudaSetDevice(e->device);
  ttx::sync_all(e);
  e->quiesced = true;  // nothing runs any more: the frees below need no further waits
  for (int li = 1; li < e->n_lanes; ++li) {
    TTLane &l = e->lanes[li];
    dfree(e, l.d_segs);
    dfree(e, l.d_tcsegs);
    dfree(e, l.d_counters);
    dfree(e, l.d_cursors);
    for (int i = 0; i < tt_engine::kSide; ++i) {
      if (l.side[i]) cudaStreamDestroy(l.side[i]);
      if (l.join[i]) cudaEventDestroy(l.join[i]);
    }
    if (l.fork) cudaEventDestroy(l.fork);
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  if (e->lane_pre) cudaEventDestroy(e->lane_pre);
  for (tt_chan *c : e->table)
    if (c) {
      dfree(e, c->d_in);
      dfree(e, c->d_out);
      dfree(e, c->d_taps);
      dfree(e, c->d_delays);
      dfree(e, c->d_chunks);
      dfree(e, c->d_amp);
      dfree(e, c->d_freq);
      dfree(e, c->d_phase);
      dfree(e, c->d_src);
      dfree(e, c->d_sparse);
      dfree(e, c->d_sparse_dly);
      c->e = nullptr;
      delete c;
    }
  for (tt_cell *cl : e->cells) {
    dfree(e, cl->d_out);
    dfree(e, cl->d_members);
    cl->e = nullptr;
    delete cl;
  }
  e->cells.clear();
  for (auto &p : e->events) cudaEventDestroy(p.second);
  for (auto ev : e->pool) cudaEventDestroy(ev);
  for (int li = 0; li < e->n_lanes; ++li)
    if (e->lanes[li].gexec) cudaGraphExecDestroy(e->lanes[li].gexec);
  dfree(e, e->d_ues);
  dfree(e, e->d_segs);
  dfree(e, e->d_gsegs);
  dfree(e, e->d_counters);
  dfree(e, e->d_cursors);
  dfree(e, e->d_tcsegs);
  dfree(e, e->d_sos);
  dfree(e, e->d_retime);
  dfree(e, e->d_topn);
  dfree(e, e->d_status);
  dfree(e, e->d_check);
  if (e->stream) cudaStreamDestroy(e->stream);
  if (e->copy) cudaStreamDestroy(e->copy);
  if (e->h2d) cudaStreamDestroy(e->h2d);
  for (int i = 0; i < tt_engine::kSide; ++i) {
    if (e->side[i]) cudaStreamDestroy(e->side[i]);
    if (e->join[i]) cudaEventDestroy(e->join[i]);
  }
  if (e->fork) cudaEventDestroy(e->fork);
  delete e;
  return TT_OK;
}

tt_status tt_engine_stream(tt_engine *e, void **stream) {
  if (!e || !stream) return fail(TT_ERR_INVALID, "null argument");
  *stream = (void *)e->stream;
  return TT_OK;
}

tt_status tt_engine_get_stats(tt_engine *e, tt_engine_stats *out) {
  if (!e || !out) return fail(TT_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(e->mu);
  tt_engine_stats s{};
  s.hbm_in_use = e->in_use;
  s.hbm_budget = e->budget;
  for (tt_chan *c : e->table) s.n_chans += c ? 1 : 0;
  s.launches = e->launches;
  s.slots_processed = e->slots_processed;
  s.graph_builds = e->graph_builds;
  s.graph_launches = e->graph_launches;
  *out = s;
  return TT_OK;
}

tt_status tt_chan_create(tt_engine *e, const tt_chan_config *cfg, tt_chan **out) {
  if (!e || !cfg || !out || cfg->struct_size < sizeof(tt_chan_config))
    return fail(TT_ERR_INVALID, "tt_chan_create: bad config");
  const uint32_t N = cfg->samples_per_slot;
  if (N == 0 || N > (1u << 24)) return fail(TT_ERR_INVALID, "samples_per_slot out of range");
  if (cfg->symbols_per_slot == 0 || cfg->symbols_per_slot > TT_MAX_SYM || !cfg->symbol_len)
    return fail(TT_ERR_INVALID, "symbols_per_slot must be 1..%d with symbol_len given", TT_MAX_SYM);
  if (cfg->n_tx < 1 || cfg->n_tx > TT_MAX_ANT || cfg->n_rx < 1 || cfg->n_rx > TT_MAX_ANT)
    return fail(TT_ERR_INVALID, "n_tx and n_rx must be 1..%d", TT_MAX_ANT);
  if (cfg->max_taps < 1 || cfg->max_taps > TT_MAX_TAPS)
    return fail(TT_ERR_INVALID, "max_taps must be 1..%d", TT_MAX_TAPS);
  if (cfg->max_delay > TT_MAX_DELAY) return fail(TT_ERR_INVALID, "max_delay must be <= %d", TT_MAX_DELAY);
  if (cfg->precision > TT_FP16_TC) return fail(TT_ERR_INVALID, "unknown precision");
  if (cfg->output_format > TT_OUT_CF32) return fail(TT_ERR_INVALID, "unknown output_format");
  if (cfg->top_n && (cfg->precision != TT_FP32 || e->form == TT_FORM_PLAIN))
    return fail(TT_ERR_INVALID, "top_n needs the FP32 batched form");
  if (!(cfg->noise_var >= 0.0f) || !std::isfinite(cfg->noise_var)) return fail(TT_ERR_INVALID, "bad noise_var");
  uint64_t sum = 0;
  for (uint32_t j = 0; j < cfg->symbols_per_slot; ++j) {
    if (cfg->symbol_len[j] == 0) return fail(TT_ERR_INVALID, "zero symbol length");
    sum += cfg->symbol_len[j];
  }
  if (sum != N) return fail(TT_ERR_INVALID, "symbol lengths sum to %llu, not %u", (unsigned long long)sum, N);
  const int hist = (int)((cfg->max_delay + N - 1) / N);
  int Q = (int)cfg->ring_slots;
  if (Q == 0) Q = hist + 4;
  if (Q < hist + 2 || Q > (1 << 20)) return fail(TT_ERR_INVALID, "ring_slots must be >= %d", hist + 2);

  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  uint32_t idx = 0;
  while (idx < e->max_ues && e->table[idx]) ++idx;
  if (idx == e->max_ues) return fail(TT_ERR_NO_MEMORY, "UE table full (%u)", e->max_ues);
  const size_t in_e = (size_t)cfg->n_tx * N * 2;
  const size_t out_e = (size_t)cfg->n_rx * N * (cfg->output_format == TT_OUT_CF32 ? 4 : 2);
  const uint64_t bytes = (uint64_t)Q * (in_e + out_e) * sizeof(int16_t);
  if (e->budget && e->in_use + bytes > e->budget)
    return fail(TT_ERR_NO_MEMORY, "admission refused: %llu B needed, %llu of %llu B in use",
                (unsigned long long)bytes, (unsigned long long)e->in_use, (unsigned long long)e->budget);
  tt_chan *c = new tt_chan();
  c->e = e;
  c->index = idx;
  c->cfg = *cfg;
  c->sym_len.assign(cfg->symbol_len, cfg->symbol_len + cfg->symbols_per_slot);
  c->cfg.symbol_len = nullptr;
  c->n = (int)N;
  c->Q = Q;
  c->hist = hist;
  c->slot_in_elems = in_e;
  c->slot_out_elems = out_e;
  cudaError_t err = dmalloc(e, &c->d_in, (size_t)Q * in_e * sizeof(int16_t));
  if (err == cudaSuccess) err = dmalloc(e, &c->d_out, (size_t)Q * out_e * sizeof(int16_t));
  if (err == cudaSuccess) err = cudaMemsetAsync(c->d_in, 0, (size_t)Q * in_e * sizeof(int16_t), e->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(c->d_out, 0, (size_t)Q * out_e * sizeof(int16_t), e->stream);
  if (err != cudaSuccess) {
    dfree(e, c->d_in);
    dfree(e, c->d_out);
    delete c;
    return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA, "ring allocation: %s",
                cudaGetErrorString(err));
  }
  c->ring_bytes = bytes;
  e->in_use += bytes;
  TTUEDesc &d = c->desc;
  d.ring_in = c->d_in;
  d.ring_out = c->d_out;
  d.n = (int)N;
  d.nsym = (int)cfg->symbols_per_slot;
  d.n_tx = (int)cfg->n_tx;
  d.n_rx = (int)cfg->n_rx;
  d.ring_q = Q;
  d.ue_id = cfg->ue_id;
  d.seed = cfg->seed;
  d.noise_std = cfg->noise_var > 0.f ? (float)std::sqrt((double)cfg->noise_var / 2.0) : 0.f;
  d.out_f32 = cfg->output_format == TT_OUT_CF32 ? 1 : 0;
  d.top_n = (int)cfg->top_n;
  const std::vector<int> cands = spt_candidates(c->sym_len, e->spt_override, cfg->n_rx, cfg->n_tx);
  tt_status sst = set_geom(c, cands.empty() ? 1 : cands[0], e->tpb_override ? (int)e->tpb_override : TT_TPB);
  if (sst != TT_OK) {
    dfree(e, c->d_in);
    dfree(e, c->d_out);
    e->in_use -= bytes;
    delete c;
    return sst;
  }
  e->table[idx] = c;
  tt_status st = upload_desc(c);
  if (st != TT_OK) return st;
  *out = c;
  return TT_OK;
}

tt_status tt_chan_destroy(tt_chan *c) {
  if (!valid_chan(c)) return fail(TT_ERR_INVALID, "null channel");
  tt_engine *e = c->e;
  std::lock_guard<std::mutex> lk(e->mu);
  if (c->cell) return fail(TT_ERR_STATE, "channel is a member of a cell: destroy the cell first");
  cudaSetDevice(e->device);
  ttx::sync_all(e);
  dfree(e, c->d_in);
  dfree(e, c->d_out);
  dfree(e, c->d_taps);
  dfree(e, c->d_delays);
  dfree(e, c->d_chunks);
  dfree(e, c->d_amp);
  dfree(e, c->d_freq);
  dfree(e, c->d_phase);
  dfree(e, c->d_src);
  dfree(e, c->d_sparse);
  dfree(e, c->d_sparse_dly);
  e->in_use -= c->ring_bytes + c->trace_bytes + c->sparse_bytes;
  e->table[c->index] = nullptr;
  e->pending.erase(std::remove(e->pending.begin(), e->pending.end(), c), e->pending.end());
  drop_graph(e);
  c->e = nullptr;
  delete c;
  ttx::admission_notify(e);  // channels waiting for budget may fit now
  return TT_OK;
}

tt_status tt_chan_push_slot(tt_chan *c, uint64_t slot, const int16_t *iq_in) {
  return tt_chan_push_slots(c, slot, 1, iq_in);
}

tt_status tt_chan_push_slot_dev(tt_chan *c, uint64_t slot, const int16_t *d_iq_in, void *stream) {
  return tt_chan_push_slots_dev(c, slot, 1, d_iq_in, stream);
}

tt_status tt_chan_pull_slot_dev(tt_chan *c, uint64_t *slot, void *d_iq_out, void *stream) {
  if (!valid_chan(c) || !slot || !d_iq_out) return fail(TT_ERR_INVALID, "tt_chan_pull_slot_dev: bad argument");
  uint64_t s;
  {
    std::lock_guard<std::mutex> lk(c->e->mu);
    s = c->pulled_end;
  }
  tt_status st = tt_chan_pull_slots_dev(c, s, 1, d_iq_out, stream);
  if (st == TT_OK) *slot = s;
  return st;
}

tt_status tt_engine_run_slot(tt_engine *e) { return tt_engine_run(e); }

// Make stream `st` wait for every queued batch that may still read the input-ring positions that
// slots [first, first + n) overwrite: they held slots [first - Q, first + n - Q), which batches
// processing up to slot first + n - Q - 1 + hist read (the delay line).  Batches complete in order,
// so waiting for the batch holding that slot covers all of them.  Engine lock held.
static cudaError_t wait_ring_readers(tt_chan *c, uint64_t first, uint32_t n, cudaStream_t st) {
  tt_engine *e = c->e;
  if (!c->started || first + n <= (uint64_t)c->Q) return cudaSuccess;
  cudaError_t q = update_completed(e);
  if (q != cudaSuccess) return q;
  update_chan(c);
  const uint64_t last_reader_slot = first + n - (uint64_t)c->Q - 1 + (uint64_t)c->hist;
  // Completed batches have left the in-flight list: if the reader is among them, nothing to wait
  // for (the first batch still in flight is a later one, which reads other positions).
  if (last_reader_slot < c->completed_end) return cudaSuccess;
  // Every in-flight batch up to the one holding that slot reads the positions (on one lane the last
  // of them would do, but batches on different lanes may complete out of order).
  for (const auto &p : c->inflight) {
    cudaEvent_t ev = event_of(e, p.second);
    if (ev) {
      cudaError_t err = cudaStreamWaitEvent(st, ev, 0);
      if (err != cudaSuccess) return err;
    }
    if (p.first > last_reader_slot) break;
  }
  return cudaSuccess;
}

// The stream waits for the batches that produce this channel's slots [.., upto) and are still in
// flight (a copy of their outputs on another stream).
static cudaError_t wait_producers(tt_chan *c, uint64_t upto, cudaStream_t st) {
  tt_engine *e = c->e;
  cudaError_t q = update_completed(e);
  if (q != cudaSuccess) return q;
  update_chan(c);
  for (const auto &p : c->inflight) {
    cudaEvent_t ev = event_of(e, p.second);
    if (ev) {
      cudaError_t err = cudaStreamWaitEvent(st, ev, 0);
      if (err != cudaSuccess) return err;
    }
    if (p.first >= upto) break;
  }
  return cudaSuccess;
}

// The per-run pre-passes (timed-trace anchors, synthesised anchors, top-n selection) rewrite a
// channel's anchor and sparse-tap rings, (Q + 1) * nsym + 1 anchors long, from the first anchor of
// slot launched_end to the first anchor of slot pushed_end.  A rewritten position last held the
// anchor one ring length earlier, read by batches holding a slot at most pushed_end - Q - 2.  On
// one stream those finished before the pre-pass started; on other launch lanes they may still run
// (replays release outputs at launch, so the host runs ahead), so the engine stream waits for
// them first.  Engine lock held.
static cudaError_t wait_anchor_readers(tt_engine *e, const std::vector<tt_chan *> &chans) {
  bool polled = false;
  for (tt_chan *c : chans) {
    if (!(c->retime || c->synth || (sparse(c) && c->d_sparse)) || c->pushed_end <= c->launched_end) continue;
    const uint64_t reach = (uint64_t)c->Q + 2;
    if (c->pushed_end < reach) continue;
    const uint64_t last = c->pushed_end - reach;  // the newest slot whose anchors may share a position
    if (!polled) {
      cudaError_t q = update_completed(e);
      if (q != cudaSuccess) return q;
      polled = true;
    }
    update_chan(c);
    uint64_t start = c->completed_end;  // first slot of the oldest batch still in flight
    for (const auto &p : c->inflight) {
      if (start > last) break;
      if (cudaEvent_t w = event_of(e, p.second)) {
        cudaError_t err = cudaStreamWaitEvent(e->stream, w, 0);
        if (err != cudaSuccess) return err;
      }
      start = p.first;
    }
  }
  return cudaSuccess;
}

tt_status tt_chan_push_slots(tt_chan *c, uint64_t first, uint32_t n, const int16_t *iq_in) {
  const ttx::NvtxScope nvtx_range("tt push (host)");
  if (!valid_chan(c) || (!iq_in && n)) return fail(TT_ERR_INVALID, "tt_chan_push_slots: bad argument");
  if (n == 0) return TT_OK;
  tt_engine *e = c->e;
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status s = check_room(c, first, n);
  if (s == TT_ERR_AGAIN && e->server) s = ttx::server_wait_room(e, lk, [&] { return check_room(c, first, n); });
  if (s != TT_OK) return s;
  // On the push stream, after any queued kernel that still reads the ring positions being
  // overwritten (others keep running), then wait, with the engine unlocked, so the caller's
  // buffer is free.  The slots count as pushed only once the copy is complete, so no kernel
  // reads them earlier.
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = wait_ring_readers(c, first, n, e->h2d);
  if (err == cudaSuccess)
    err = ring_copy(c->d_in, c->slot_in_elems, c->Q, first, n, iq_in, nullptr, cudaMemcpyHostToDevice, e->h2d, true);
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->h2d);
  if (err == cudaSuccess) {
    lk.unlock();
    err = cudaEventSynchronize(ev);
    lk.lock();
  }
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "push copy: %s", cudaGetErrorString(err));
  mark_pushed(c, first, n);
  if (e->server) e->work_cv.notify_one();
  return TT_OK;
}

tt_status tt_engine_push_slots(tt_engine *e, uint32_t n_chans, tt_chan *const *chans, const uint64_t *first,
                               const uint32_t *n, const int16_t *const *iq_in) {
  if (!e || (n_chans && (!chans || !first || !n || !iq_in))) return fail(TT_ERR_INVALID, "tt_engine_push_slots: bad argument");
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  for (uint32_t i = 0; i < n_chans; ++i) {
    tt_chan *c = chans[i];
    if (!valid_chan(c) || c->e != e || (n[i] && !iq_in[i])) return fail(TT_ERR_INVALID, "push entry %u: bad channel or buffer", i);
    for (uint32_t j = 0; j < i; ++j)
      if (chans[j] == c) return fail(TT_ERR_INVALID, "push entry %u: channel repeated", i);
    tt_status s = check_room(c, first[i], n[i]);
    if (s == TT_ERR_AGAIN && e->server)
      s = ttx::server_wait_room(e, lk, [&] { return check_room(c, first[i], n[i]); });
    if (s != TT_OK) return s;
  }
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = cudaSuccess;
  for (uint32_t i = 0; i < n_chans && err == cudaSuccess; ++i) {
    if (!n[i]) continue;
    tt_chan *c = chans[i];
    err = wait_ring_readers(c, first[i], n[i], e->h2d);
    if (err == cudaSuccess)
      err = ring_copy(c->d_in, c->slot_in_elems, c->Q, first[i], n[i], iq_in[i], nullptr, cudaMemcpyHostToDevice,
                      e->h2d, true);
  }
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->h2d);
  if (err == cudaSuccess) {
    lk.unlock();
    err = cudaEventSynchronize(ev);
    lk.lock();
  }
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "push copy: %s", cudaGetErrorString(err));
  for (uint32_t i = 0; i < n_chans; ++i)
    if (n[i]) mark_pushed(chans[i], first[i], n[i]);
  if (e->server) e->work_cv.notify_one();
  return TT_OK;
}

tt_status tt_chan_push_slots_dev(tt_chan *c, uint64_t first, uint32_t n, const int16_t *d_iq_in,
                                 void *stream) {
  const ttx::NvtxScope nvtx_range("tt push (device)");
  if (!valid_chan(c) || (!d_iq_in && n)) return fail(TT_ERR_INVALID, "tt_chan_push_slots_dev: bad argument");
  if (n == 0) return TT_OK;
  tt_engine *e = c->e;
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status s = check_room(c, first, n);
  if (s == TT_ERR_AGAIN && e->server) s = ttx::server_wait_room(e, lk, [&] { return check_room(c, first, n); });
  if (s != TT_OK) return s;
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = cudaEventRecord(ev, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, ev, 0);
  if (err == cudaSuccess) err = wait_ring_readers(c, first, n, e->stream);  // batches on other lanes
  if (err == cudaSuccess)
    err = ring_copy(c->d_in, c->slot_in_elems, c->Q, first, n, d_iq_in, nullptr, cudaMemcpyDeviceToDevice,
                    e->stream, true);
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "push copy: %s", cudaGetErrorString(err));
  mark_pushed(c, first, n);
  if (e->server) e->work_cv.notify_one();
  return TT_OK;
}

tt_status tt_chan_slot_input(tt_chan *c, uint64_t slot, int16_t **d_ptr) {
  if (!valid_chan(c) || !d_ptr) return fail(TT_ERR_INVALID, "tt_chan_slot_input: bad argument");
  std::lock_guard<std::mutex> lk(c->e->mu);
  const uint64_t start = c->started ? c->pulled_end : slot;
  if (c->started && slot < c->pushed_end) return fail(TT_ERR_STATE, "slot %llu already pushed",
                                                      (unsigned long long)slot);
  if (slot + 1 - start + (uint64_t)c->hist > (uint64_t)c->Q) return fail(TT_ERR_AGAIN, "slot ring full");
  *d_ptr = c->d_in + (size_t)(slot % (uint64_t)c->Q) * c->slot_in_elems;
  return TT_OK;
}

tt_status tt_chan_commit_slots(tt_chan *c, uint64_t first, uint32_t n) {
  const ttx::NvtxScope nvtx_range("tt commit");
  if (!valid_chan(c)) return fail(TT_ERR_INVALID, "null channel");
  if (n == 0) return TT_OK;
  tt_engine *e = c->e;
  std::unique_lock<std::mutex> lk(e->mu);
  tt_status s = check_room(c, first, n);
  if (s == TT_ERR_AGAIN && e->server) s = ttx::server_wait_room(e, lk, [&] { return check_room(c, first, n); });
  if (s != TT_OK) return s;
  mark_pushed(c, first, n);
  if (e->server) e->work_cv.notify_one();
  return TT_OK;
}

tt_status tt_engine_run(tt_engine *e) {
  const ttx::NvtxScope nvtx_range("tt run");
  if (!e) return fail(TT_ERR_INVALID, "null engine");
  std::lock_guard<std::mutex> lk(e->mu);
  if (e->server && !ttx::is_server_thread(e))
    return fail(TT_ERR_STATE, "a server is running on this engine: it launches the pushed slots itself");
  TT_CK(cudaSetDevice(e->device));
  if (tt_checked_build()) {  // bounds-checked build, tests only: lower the output-store bound
    const char *v = std::getenv("TT_TEST_CHECK_SHRINK");
    e->check_shrink = v ? std::atoi(v) : 0;
  }
  std::vector<tt_chan *> ready, tc_ready;
  // the channels with unlaunched slots, in table order (the order the plan and a cached graph use)
  std::sort(e->pending.begin(), e->pending.end(), [](const tt_chan *a, const tt_chan *b) { return a->index < b->index; });
  for (tt_chan *c : e->pending)
    if (c->has_trace && c->started && c->pushed_end > c->launched_end) {
      if (c->cfg.precision != TT_FP32 && e->form != TT_FORM_PLAIN) tc_ready.push_back(c);
      else ready.push_back(c);
    }
  if (ready.empty() && tc_ready.empty() && e->cells.empty()) return TT_OK;
  // the batch's completion event is taken before anything launches, so whatever launches below
  // is always registered
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  struct EventGuard {
    tt_engine *e;
    cudaEvent_t ev;
    ~EventGuard() {
      if (ev) e->pool.push_back(ev);
    }
  } guard{e, ev};
  {  // anchor and sparse-tap pre-passes, on the engine stream
    std::vector<tt_chan *> all(ready);
    all.insert(all.end(), tc_ready.begin(), tc_ready.end());
    TT_CK(wait_anchor_readers(e, all));
    tt_status sst = ttx::launch_retime(e, all);
    if (sst == TT_OK) sst = ttx::launch_synth(e, all);
    if (sst == TT_OK) sst = ttx::launch_topn(e, ready);
    if (sst != TT_OK) return sst;
  }
  // The batch's lane: while a server runs or graphs are replayed, batches rotate over the lanes so
  // that consecutive ones overlap on the GPU.  Not with cells: a cell's aggregation frees its
  // members' output slots when it is launched, so a later batch must not start before it ends.  A lane other than the engine stream
  // first waits for everything queued there (device pushes and pulls, descriptor uploads, the
  // pre-passes above).
  const int rot = rotation(e);
  const int li = rot > 1 ? (int)((e->launch_seq + 1) % (uint64_t)rot) : 0;
  TTLane &ln = e->lanes[li];
  if (li != 0) {
    TT_CK(cudaEventRecord(e->lane_pre, e->stream));
    TT_CK(cudaStreamWaitEvent(ln.stream, e->lane_pre, 0));
  }
  if (rot > 1) {
    // Output slots released before their batch completed (tt_chan_release_slots, replays) may be
    // rewritten by this batch while that batch, on another lane, still writes them: wait for it.
    // One stream ordered such writes by itself.
    TT_CK(update_completed(e));
    std::vector<uint64_t> seqs;
    for (const std::vector<tt_chan *> *list : {&ready, &tc_ready})
      for (tt_chan *c : *list) {
        update_chan(c);
        const uint64_t bound = c->pushed_end > (uint64_t)c->Q ? c->pushed_end - (uint64_t)c->Q : 0;
        uint64_t start = c->completed_end;
        for (const auto &p : c->inflight) {
          if (start >= bound) break;
          seqs.push_back(p.second);
          start = p.first;
        }
      }
    std::sort(seqs.begin(), seqs.end());
    seqs.erase(std::unique(seqs.begin(), seqs.end()), seqs.end());
    for (uint64_t q : seqs)
      if (cudaEvent_t w = event_of(e, q)) TT_CK(cudaStreamWaitEvent(ln.stream, w, 0));
  }
  if (e->server) {  // the batch's first device-side moment, for the server's GPU-time statistics
    tt_status sst = ttx::server_stamp_start(e, e->launch_seq + 1, ln.stream);
    if (sst != TT_OK) return sst;
  }

  if (e->form == TT_FORM_PLAIN) {
    for (tt_chan *c : ready) {
      for (uint64_t s = c->launched_end; s < c->pushed_end; ++s) {
        cudaError_t err = tt_launch_plain(e->d_ues + c->index, s, c->n, ln.stream);
        if (err != cudaSuccess) return fail(TT_ERR_CUDA, "plain launch: %s", cudaGetErrorString(err));
        ++e->launches;
      }
    }
  } else if (!ready.empty()) {
    std::vector<uint64_t> first(ready.size()), count(ready.size());
    for (size_t i = 0; i < ready.size(); ++i) {
      first[i] = ready[i]->launched_end;
      count[i] = ready[i]->pushed_end - ready[i]->launched_end;
    }
    if (e->graphs && !e->gkey.empty() && e->gstride == rot && ln.gexec && ready == e->gchans &&
        count == e->gcounts) {
      // same channels, same slots per run: replay without re-planning
      std::vector<tt_chan *> &seg_chans = e->gplan_chans;
      for (size_t i = 0; i < seg_chans.size(); ++i) e->gsegs_host[i].first_slot = seg_chans[i]->launched_end;
      tt_status st = launch_cached_graph(e, seg_chans, e->gsegs_host, li);
      if (st != TT_OK) return st;
    } else {
      Plan plan;
      tt_status st = build_plan(e, ready, first, count, plan);
      if (st != TT_OK) return st;
      st = e->graphs ? launch_graph(e, plan, li) : launch_direct(e, plan, ln);
      if (st != TT_OK) return st;
      if (e->graphs) {
        e->gchans = ready;
        e->gcounts = count;
        e->gplan_chans = plan.chans;
      }
    }
  }
  if (!tc_ready.empty()) {
    tt_status st = launch_tc(e, tc_ready, ln);
    if (st != TT_OK) return st;
    ready.insert(ready.end(), tc_ready.begin(), tc_ready.end());
  }
  std::vector<uint64_t> prev_end(ready.size());
  for (size_t i = 0; i < ready.size(); ++i) {
    prev_end[i] = ready[i]->launched_end;
    ready[i]->launched_end = ready[i]->pushed_end;
  }
  {  // channels still holding unlaunched slots (no trace yet) stay listed
    size_t k = 0;
    for (tt_chan *c : e->pending) {
      if (c->pushed_end > c->launched_end) e->pending[k++] = c;
      else c->in_pending = false;
    }
    e->pending.resize(k);
  }
  // uplink aggregation of every slot all members of a cell have launched (after their kernels);
  // a failure here still registers the channels' launched slots before it is reported
  std::vector<std::pair<tt_cell *, uint64_t>> cell_ends;
  const tt_status cst = ttx::launch_cells(e, cell_ends);
  if (ready.empty() && cell_ends.empty()) return cst;
  if (e->server) {
    tt_status sst = ttx::server_stamp(e, e->launch_seq + 1, ln.stream);
    if (sst != TT_OK) return sst;
  }
  TT_CK(cudaEventRecord(ev, ln.stream));
  guard.ev = nullptr;  // owned by the batch list from here on
  const uint64_t seq = ++e->launch_seq;
  ln.last_seq = seq;
  e->events.emplace_back(seq, ev);
  for (size_t i = 0; i < ready.size(); ++i) {
    e->slots_processed += ready[i]->launched_end - prev_end[i];
    ready[i]->inflight.emplace_back(ready[i]->launched_end, seq);
    if (e->server) ttx::server_note_launch(ready[i], prev_end[i], ready[i]->launched_end, seq);
  }
  for (auto &ce : cell_ends) {
    tt_cell *cl = ce.first;
    cl->inflight.emplace_back(ce.second, seq);
    cl->launched_end = ce.second;
    for (tt_chan *m : cl->members) m->pulled_end = std::max(m->pulled_end, ce.second);  // consumed
  }
  return cst;
}

tt_status tt_engine_replay(tt_engine *e, uint32_t n_steps, uint32_t slots_per_step) {
  const ttx::NvtxScope nvtx_range("tt replay");
  if (!e || slots_per_step == 0) return fail(TT_ERR_INVALID, "tt_engine_replay: bad argument");
  for (uint32_t step = 0; step < n_steps; ++step) {
    {
      std::lock_guard<std::mutex> lk(e->mu);
      for (tt_chan *c : e->table) {
        if (!c || !c->has_trace || !c->started) continue;
        // release what the previous steps produced, then reuse the ring in place
        c->pulled_end = std::max(c->pulled_end, std::min(c->launched_end, c->pushed_end));
      }
      for (tt_cell *cl : e->cells) cl->pulled_end = std::max(cl->pulled_end, cl->launched_end);
      for (tt_chan *c : e->table) {
        if (!c || !c->has_trace || !c->started) continue;
        tt_status st = check_room(c, c->pushed_end, slots_per_step);
        if (st != TT_OK) return st;
        mark_pushed(c, c->pushed_end, slots_per_step);
      }
    }
    tt_status st = tt_engine_run(e);
    if (st != TT_OK) return st;
  }
  return TT_OK;
}

tt_status tt_engine_sync(tt_engine *e, int64_t timeout_us) {
  if (!e) return fail(TT_ERR_INVALID, "null engine");
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status s = wait_seq(e, e->launch_seq, timeout_us, lk);
  if (s != TT_OK) return s;
  if (timeout_us < 0) ttx::sync_all(e);
  int kst = 0;
  TT_CK(cudaMemcpy(&kst, e->d_status, sizeof kst, cudaMemcpyDeviceToHost));
  if (kst) {
    cudaMemset(e->d_status, 0, sizeof(int));
    cudaStreamSynchronize(nullptr);  // landed before the next run's kernels can set it again
    return fail(TT_ERR_TIMEOUT, "a kernel's bounded wait on the tensor core expired; its slots are invalid");
  }
  for (tt_chan *c : e->table)
    if (c) update_chan(c);
  return TT_OK;
}

tt_status tt_engine_join(tt_engine *e) {
  if (!e) return fail(TT_ERR_INVALID, "null engine");
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  for (const auto &p : e->events)  // batches not yet seen complete (the others are done)
    TT_CK(cudaStreamWaitEvent(e->stream, p.second, 0));
  return TT_OK;
}

tt_status tt_engine_get_check(tt_engine *e, tt_check_report *out) {
  if (!e || !out) return fail(TT_ERR_INVALID, "null engine or output");
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status s = wait_seq(e, e->launch_seq, -1, lk);
  if (s != TT_OK) return s;
  ttx::sync_all(e);
  uint32_t w[2] = {0, 0};
  TT_CK(cudaMemcpy(w, e->d_check, sizeof w, cudaMemcpyDeviceToHost));
  TT_CK(cudaMemset(e->d_check, 0, sizeof w));
  TT_CK(cudaStreamSynchronize(nullptr));  // landed before the next run's kernels count again
  tt_check_report r{};
  r.checked_build = (uint32_t)tt_checked_build();
  r.violations = w[0];
  r.first_code = w[1];
  *out = r;
  return TT_OK;
}

static tt_status pull_common(tt_chan *c, uint64_t first, uint32_t n, void *out, int64_t timeout_us) {
  const ttx::NvtxScope nvtx_range("tt pull");
  tt_engine *e = c->e;
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  if (c->cell) return fail(TT_ERR_STATE, "the channel's outputs go to its cell");
  if (!c->started) return fail(TT_ERR_AGAIN, "nothing pushed to this channel yet");
  if (first != c->pulled_end)
    return fail(TT_ERR_STATE, "pull must start at the oldest unpulled slot %llu", (unsigned long long)c->pulled_end);
  if (first + n > c->launched_end) return fail(TT_ERR_AGAIN, "slot not launched yet");
  update_chan(c);
  if (first + n > c->completed_end) {
    uint64_t need = 0;
    for (auto &p : c->inflight)
      if (p.first >= first + n) { need = p.second; break; }
    tt_status s = wait_seq(e, need, timeout_us, lk);
    if (s != TT_OK) return s;
    update_chan(c);
  }
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = ring_copy(c->d_out, c->slot_out_elems, c->Q, first, n, nullptr, out,
                              cudaMemcpyDeviceToHost, e->copy, false);
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->copy);
  if (err == cudaSuccess) {  // wait for the copy with the engine unlocked (a pusher may run meanwhile)
    lk.unlock();
    err = cudaEventSynchronize(ev);
    lk.lock();
  }
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "pull copy: %s", cudaGetErrorString(err));
  c->pulled_end = first + n;
  return TT_OK;
}

tt_status tt_engine_pull_slots(tt_engine *e, uint32_t n_chans, tt_chan *const *chans, const uint64_t *first,
                               const uint32_t *n, void *const *iq_out, int64_t timeout_us) {
  if (!e || (n_chans && (!chans || !first || !n || !iq_out))) return fail(TT_ERR_INVALID, "tt_engine_pull_slots: bad argument");
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  uint64_t need = 0;  // the batch that completes the last requested slot of every entry
  for (uint32_t i = 0; i < n_chans; ++i) {
    tt_chan *c = chans[i];
    if (!valid_chan(c) || c->e != e || (n[i] && !iq_out[i])) return fail(TT_ERR_INVALID, "pull entry %u: bad channel or buffer", i);
    if (c->cell) return fail(TT_ERR_STATE, "pull entry %u: the channel's outputs go to its cell", i);
    for (uint32_t j = 0; j < i; ++j)
      if (chans[j] == c) return fail(TT_ERR_INVALID, "pull entry %u: channel repeated", i);
    if (!n[i]) continue;
    if (!c->started || first[i] != c->pulled_end)
      return fail(TT_ERR_STATE, "pull entry %u must start at the oldest unpulled slot %llu", i,
                  (unsigned long long)c->pulled_end);
    if (first[i] + n[i] > c->launched_end) return fail(TT_ERR_AGAIN, "pull entry %u: slot not launched yet", i);
    update_chan(c);
    if (first[i] + n[i] > c->completed_end)
      for (auto &p : c->inflight)
        if (p.first >= first[i] + n[i]) { need = std::max(need, p.second); break; }
  }
  if (need) {
    tt_status s = wait_seq(e, need, timeout_us, lk);
    if (s != TT_OK) return s;
  }
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = cudaSuccess;
  for (uint32_t i = 0; i < n_chans && err == cudaSuccess; ++i)
    if (n[i])
      err = ring_copy(chans[i]->d_out, chans[i]->slot_out_elems, chans[i]->Q, first[i], n[i], nullptr, iq_out[i],
                      cudaMemcpyDeviceToHost, e->copy, false);
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->copy);
  if (err == cudaSuccess) {
    lk.unlock();
    err = cudaEventSynchronize(ev);
    lk.lock();
  }
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "pull copy: %s", cudaGetErrorString(err));
  for (uint32_t i = 0; i < n_chans; ++i)
    if (n[i]) chans[i]->pulled_end = first[i] + n[i];
  return TT_OK;
}

tt_status tt_chan_pull_slot(tt_chan *c, uint64_t *slot, void *iq_out, int64_t timeout_us) {
  if (!valid_chan(c) || !slot || !iq_out) return fail(TT_ERR_INVALID, "tt_chan_pull_slot: bad argument");
  uint64_t s;
  {
    std::lock_guard<std::mutex> lk(c->e->mu);
    s = c->pulled_end;
  }
  tt_status st = pull_common(c, s, 1, iq_out, timeout_us);
  if (st == TT_OK) *slot = s;
  return st;
}

tt_status tt_chan_pull_slots(tt_chan *c, uint64_t first, uint32_t n, void *iq_out, int64_t timeout_us) {
  if (!valid_chan(c) || (!iq_out && n)) return fail(TT_ERR_INVALID, "tt_chan_pull_slots: bad argument");
  if (n == 0) return TT_OK;
  return pull_common(c, first, n, iq_out, timeout_us);
}

tt_status tt_chan_pull_slots_dev(tt_chan *c, uint64_t first, uint32_t n, void *d_iq_out, void *stream) {
  if (!valid_chan(c) || (!d_iq_out && n)) return fail(TT_ERR_INVALID, "tt_chan_pull_slots_dev: bad argument");
  if (n == 0) return TT_OK;
  tt_engine *e = c->e;
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  if (c->cell) return fail(TT_ERR_STATE, "the channel's outputs go to its cell");
  if (!c->started) return fail(TT_ERR_AGAIN, "nothing pushed to this channel yet");
  if (first != c->pulled_end)
    return fail(TT_ERR_STATE, "pull must start at the oldest unpulled slot %llu", (unsigned long long)c->pulled_end);
  if (first + n > c->launched_end) return fail(TT_ERR_AGAIN, "slot not launched yet");
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = wait_producers(c, first + n, e->stream);  // batches on other lanes
  if (err == cudaSuccess)
    err = ring_copy(c->d_out, c->slot_out_elems, c->Q, first, n, nullptr, d_iq_out, cudaMemcpyDeviceToDevice,
                    e->stream, false);
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent((cudaStream_t)stream, ev, 0);
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "pull copy: %s", cudaGetErrorString(err));
  c->pulled_end = first + n;
  return TT_OK;
}

tt_status tt_chan_slot_output(tt_chan *c, uint64_t slot, const void **d_ptr) {
  if (!valid_chan(c) || !d_ptr) return fail(TT_ERR_INVALID, "tt_chan_slot_output: bad argument");
  std::lock_guard<std::mutex> lk(c->e->mu);
  if (!c->started || slot < c->pulled_end || slot >= c->launched_end)
    return fail(TT_ERR_STATE, "slot %llu is not a launched, unreleased slot", (unsigned long long)slot);
  *d_ptr = c->d_out + (size_t)(slot % (uint64_t)c->Q) * c->slot_out_elems;
  return TT_OK;
}

tt_status tt_chan_release_slots(tt_chan *c, uint64_t first, uint32_t n) {
  if (!valid_chan(c)) return fail(TT_ERR_INVALID, "null channel");
  std::lock_guard<std::mutex> lk(c->e->mu);
  if (c->cell) return fail(TT_ERR_STATE, "the channel's outputs go to its cell");
  if (!c->started || first != c->pulled_end || first + n > c->launched_end)
    return fail(TT_ERR_STATE, "release must cover launched slots from %llu", (unsigned long long)c->pulled_end);
  c->pulled_end = first + n;
  return TT_OK;
}

// ---- checkpoint / resume ----
namespace {
struct StateHeader {
  uint32_t magic;  // 'TTS1'
  uint32_t version;
  uint32_t n, n_tx, hist_samples, started;
  uint64_t next_slot, seed;
  uint32_t ue_id, pad;
};
const uint32_t kStateMagic = 0x31535454u;
}  // namespace

tt_status tt_chan_get_state(const tt_chan *cc, void *buf, size_t *len) {
  tt_chan *c = const_cast<tt_chan *>(cc);
  if (!valid_chan(c) || !len) return fail(TT_ERR_INVALID, "tt_chan_get_state: bad argument");
  const uint32_t D = c->cfg.max_delay;
  const size_t need = sizeof(StateHeader) + (size_t)c->cfg.n_tx * D * 2 * sizeof(int16_t);
  if (!buf) {
    *len = need;
    return TT_OK;
  }
  if (*len < need) return fail(TT_ERR_INVALID, "state buffer too small (%zu < %zu)", *len, need);
  tt_engine *e = c->e;
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  cudaError_t q = update_completed(e);
  if (q != cudaSuccess) return fail(TT_ERR_CUDA, "%s", cudaGetErrorString(q));
  update_chan(c);
  if (c->launched_end != c->pushed_end || c->completed_end != c->launched_end)
    return fail(TT_ERR_STATE, "channel has pending or running slots; run and sync first");
  ttx::sync_all(e);
  StateHeader h{};
  h.magic = kStateMagic;
  h.version = 1;
  h.n = (uint32_t)c->n;
  h.n_tx = c->cfg.n_tx;
  h.hist_samples = D;
  h.started = c->started ? 1u : 0u;
  h.next_slot = c->pushed_end;
  h.seed = c->cfg.seed;
  h.ue_id = c->cfg.ue_id;
  std::memcpy(buf, &h, sizeof h);
  int16_t *out = reinterpret_cast<int16_t *>(static_cast<char *>(buf) + sizeof h);
  std::memset(out, 0, (size_t)c->cfg.n_tx * D * 2 * sizeof(int16_t));
  if (c->started) {
    // samples m in [next*N - D, next*N) of every Tx antenna, from the ring slots holding them
    const uint64_t next = c->pushed_end;
    std::vector<int16_t> slotbuf(c->slot_in_elems);
    for (int b = c->hist; b >= 1; --b) {
      if ((uint64_t)b > next) continue;
      const uint64_t s = next - (uint64_t)b;
      TT_CK(cudaMemcpy(slotbuf.data(), c->d_in + (size_t)(s % (uint64_t)c->Q) * c->slot_in_elems,
                       c->slot_in_elems * sizeof(int16_t), cudaMemcpyDeviceToHost));
      for (uint32_t t = 0; t < c->cfg.n_tx; ++t)
        for (uint32_t i = 0; i < D; ++i) {
          const int64_t m = (int64_t)next * c->n - (int64_t)D + (int64_t)i;
          if (m < (int64_t)s * c->n || m >= (int64_t)(s + 1) * c->n) continue;
          const size_t w = (size_t)(m - (int64_t)s * c->n);
          out[((size_t)t * D + i) * 2] = slotbuf[((size_t)t * c->n + w) * 2];
          out[((size_t)t * D + i) * 2 + 1] = slotbuf[((size_t)t * c->n + w) * 2 + 1];
        }
    }
  }
  *len = need;
  return TT_OK;
}

tt_status tt_chan_set_state(tt_chan *c, const void *buf, size_t len) {
  if (!valid_chan(c) || !buf) return fail(TT_ERR_INVALID, "tt_chan_set_state: bad argument");
  StateHeader h{};
  if (len < sizeof h) return fail(TT_ERR_STATE, "state blob too short");
  std::memcpy(&h, buf, sizeof h);
  const uint32_t D = c->cfg.max_delay;
  if (h.magic != kStateMagic || h.version != 1 || h.n != (uint32_t)c->n || h.n_tx != c->cfg.n_tx ||
      h.hist_samples != D || len < sizeof h + (size_t)h.n_tx * D * 2 * sizeof(int16_t))
    return fail(TT_ERR_STATE, "state blob does not match this channel");
  tt_engine *e = c->e;
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  cudaError_t q = update_completed(e);
  if (q != cudaSuccess) return fail(TT_ERR_CUDA, "%s", cudaGetErrorString(q));
  update_chan(c);
  if (c->launched_end != c->pushed_end || c->completed_end != c->launched_end)
    return fail(TT_ERR_STATE, "channel has pending or running slots");
  ttx::sync_all(e);
  const int16_t *in = reinterpret_cast<const int16_t *>(static_cast<const char *>(buf) + sizeof h);
  const uint64_t next = h.next_slot;
  // zero the history slots, then write the saved samples into them
  for (int b = 1; b <= c->hist; ++b) {
    if ((uint64_t)b > next) break;
    const uint64_t s = next - (uint64_t)b;
    TT_CK(cudaMemset(c->d_in + (size_t)(s % (uint64_t)c->Q) * c->slot_in_elems, 0,
                     c->slot_in_elems * sizeof(int16_t)));
  }
  if (h.started) {
    std::vector<int16_t> slotbuf(c->slot_in_elems);
    for (int b = c->hist; b >= 1; --b) {
      if ((uint64_t)b > next) continue;
      const uint64_t s = next - (uint64_t)b;
      std::fill(slotbuf.begin(), slotbuf.end(), 0);
      for (uint32_t t = 0; t < c->cfg.n_tx; ++t)
        for (uint32_t i = 0; i < D; ++i) {
          const int64_t m = (int64_t)next * c->n - (int64_t)D + (int64_t)i;
          if (m < (int64_t)s * c->n || m >= (int64_t)(s + 1) * c->n) continue;
          const size_t w = (size_t)(m - (int64_t)s * c->n);
          slotbuf[((size_t)t * c->n + w) * 2] = in[((size_t)t * D + i) * 2];
          slotbuf[((size_t)t * c->n + w) * 2 + 1] = in[((size_t)t * D + i) * 2 + 1];
        }
      TT_CK(cudaMemcpy(c->d_in + (size_t)(s % (uint64_t)c->Q) * c->slot_in_elems, slotbuf.data(),
                       c->slot_in_elems * sizeof(int16_t), cudaMemcpyHostToDevice));
    }
  }
  // A device memset and a copy from pageable memory may return before their writes land, and the
  // engine's non-blocking streams are not ordered after the default stream: finish them here.
  TT_CK(cudaStreamSynchronize(nullptr));
  c->cfg.seed = h.seed;
  c->cfg.ue_id = h.ue_id;
  c->desc.seed = h.seed;
  c->desc.ue_id = h.ue_id;
  c->started = h.started != 0;
  c->pushed_end = c->launched_end = c->completed_end = c->pulled_end = next;
  c->inflight.clear();
  return upload_desc(c);
}

}  // extern "C"

