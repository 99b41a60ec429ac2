// Internal state of the channel engine (host side), shared by the engine's translation units:
// tt_engine.cpp (the C ABI of channels, runs and copies), tt_traces.cpp (trace loading and the
// per-run anchor pre-passes), tt_cells.cpp (uplink cells),
// tt_server.cpp (serving: the batching thread, request latencies, admission waiting list) and
// tt_tune.cpp (the autotuner and its on-disk cache).  Not part of the public ABI.
#pragma once

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "tt_chan.h"
#include "tt_internal.h"

struct TTServer;  // defined in tt_server.cpp

struct tt_chan;

struct tt_cell;

// One launch lane: the streams, events and device work lists a batch launches with.  Lane 0 is the
// engine's own stream and lists.  While a serving thread runs, or when the engine replays CUDA
// graphs, and the engine has no uplink cells, consecutive batches rotate over the lanes, so one
// batch's kernels overlap the tail and the set-up of the previous ones.  Each lane keeps its own
// instance of the cached graph and its own device slot cursors.
struct TTLane {
  static constexpr int kSide = 3;
  cudaStream_t stream = nullptr;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  TTSeg *d_segs = nullptr;         // tiled-kernel work list (max_ues entries)
  unsigned long long *d_cursors = nullptr;  // graph replay: next slot of every UE table entry on this lane
  cudaGraphExec_t gexec = nullptr;          // this lane's instance of the cached graph (shape gkey)
  TTSeg *d_tcsegs = nullptr;       // tensor-core work list (max_ues entries)
  uint32_t *d_counters = nullptr;  // one work counter per kernel variant (counter_cap)
  uint64_t last_seq = 0;           // the last batch launched on this lane
};

struct tt_engine {
  int device = 0;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  uint32_t form = TT_FORM_BATCHED;
  uint32_t max_ues = 1024;
  // allocator hook (tt_engine_config.dev_alloc/dev_free); null: cudaMalloc/cudaFree
  void *(*alloc_fn)(size_t, void *) = nullptr;
  void (*free_fn)(void *, void *) = nullptr;
  void *alloc_ctx = nullptr;
  bool quiesced = false;  // being destroyed, every stream idle
  uint32_t spt_override = 0;
  uint32_t tpb_override = 0;  // tiled kernel's threads per CTA forced for every channel (0: 128 or tuned)
  uint32_t persistent = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;  // all compute and device copies, in order
  cudaStream_t copy = nullptr;    // host pulls
  cudaStream_t h2d = nullptr;     // host pushes: wait only for kernels that still read the overwritten ring slots
  // Kernel variants of one run go on parallel branches (side streams forked from and joined
  // back to `stream`), so each variant's tail overlaps the others' work.
  static constexpr int kSide = TTLane::kSide;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  std::mutex mu;
  std::vector<tt_chan *> table;   // UE table slot -> channel
  TTUEDesc *d_ues = nullptr;
  TTSeg *d_segs = nullptr;
  size_t seg_cap = 0;
  uint32_t *d_counters = nullptr;  // one work counter per launch class
  int counter_cap = 64;
  uint64_t launch_seq = 0;         // batches issued
  uint64_t completed_seq = 0;      // batches known complete
  std::deque<std::pair<uint64_t, cudaEvent_t>> events;  // (seq, event) not yet known complete
  std::vector<cudaEvent_t> pool;
  uint64_t launches = 0, slots_processed = 0;
  // CUDA-graph replay of the batched launch (tt_engine_config.graphs)
  bool graphs = false;
  unsigned long long *d_cursors = nullptr;  // device-resident next slot of every UE table entry
  TTSeg *d_gsegs = nullptr;                 // work list owned by the cached graph
  size_t gseg_cap = 0;
  std::vector<uint64_t> gkey;               // shape of the cached graph (one instance per lane)
  int gstride = 1;                          // lanes the cached graph's replays rotate over
  std::vector<tt_chan *> gchans;            // channels of the cached graph, in table order
  std::vector<uint64_t> gcounts;            // their slots per run
  std::vector<tt_chan *> gplan_chans;       // the same channels in the graph's segment order
  uint64_t graph_builds = 0, graph_launches = 0;
  uint64_t graph_nodes = 0;                 // tiled-kernel launches inside the cached graph
  TTSeg *d_tcsegs = nullptr;                // work list of the tensor-core channels
  size_t tcseg_cap = 0;
  int *d_status = nullptr;                  // set by a kernel whose bounded wait expired
  uint32_t *d_check = nullptr;              // bounds-checked build: {violations, first code}
  int check_shrink = 0;                     // tests only (TT_TEST_CHECK_SHRINK at a run, checked build)
  int tc_no_mma = 0;                        // tests only (TT_TEST_TC_NO_MMA=1 at a run): no MMA is issued
  std::vector<TTSeg> gsegs_host;            // the cached graph's work list (first_slot refreshed per replay)
  std::vector<tt_cell *> cells;             // uplink aggregation cells
  std::vector<TTSosJob> sos_jobs;           // synthesis work list of the current run (host copy)
  TTSosJob *d_sos = nullptr;                // and its device copy
  size_t sos_cap = 0;
  std::vector<TTRetimeJob> retime_jobs;     // timed-trace anchor work list of the current run
  TTRetimeJob *d_retime = nullptr;
  size_t retime_cap = 0;
  std::vector<TTTopnJob> topn_jobs;         // tap-selection work list of the current run
  TTTopnJob *d_topn = nullptr;
  size_t topn_cap = 0;
  // serving (tt_server_start): the batching thread's state, null when no server runs
  TTServer *server = nullptr;
  std::condition_variable room_cv;          // a batch completed: ring room may have freed up
  std::condition_variable work_cv;          // a push arrived: the server may launch
  // admission waiting list (tt_chan_create_queued): tickets in arrival order
  std::mutex admit_mu;
  std::condition_variable admit_cv;
  std::deque<uint64_t> admit_queue;
  uint64_t admit_next = 0;
  // channels with pushed slots not launched yet (each once), so a run looks at those only
  std::vector<tt_chan *> pending;
  // launch lanes: lanes[0] mirrors stream/side/fork/join/d_segs/d_tcsegs/d_counters/d_cursors;
  // lanes 1.. are created with a graph-replaying engine and when a serving thread starts
  static constexpr int kLanes = 8;
  TTLane lanes[kLanes];
  int n_lanes = 1;
  cudaEvent_t lane_pre = nullptr;  // recorded on `stream` before a batch on another lane starts
  // tuning cache: class key -> (samples per thread, threads per CTA) for this device model, loaded
  // from the file TT_TUNE_CACHE names at creation and written back by the autotuner
  std::mutex tune_mu;
  std::string dev_name;
  std::string tune_path;
  std::map<std::string, std::pair<int, int>> tune;
};

struct tt_chan {
  tt_engine *e = nullptr;
  uint32_t index = 0;
  tt_chan_config cfg{};
  std::vector<uint32_t> sym_len;
  int n = 0, Q = 0, hist = 0;
  size_t slot_in_elems = 0, slot_out_elems = 0;  // int16 values per slot
  int16_t *d_in = nullptr, *d_out = nullptr;
  uint64_t ring_bytes = 0;
  float2 *d_taps = nullptr;
  int32_t *d_delays = nullptr;
  uint64_t trace_bytes = 0;
  bool has_trace = false;
  int spt = 1, tpb = TT_TPB, dclass = 0, max_sym_touched = 1;
  int32_t *d_chunks = nullptr;  // per work item of a slot: first symbol | symbols touched << 16
  int tap_need = 0;             // max symbols touched x n_rx x n_tx x K
  size_t smem = 0;
  TTUEDesc desc{};
  bool started = false;
  uint64_t pushed_end = 0, launched_end = 0, completed_end = 0, pulled_end = 0;
  uint64_t start_slot = 0;           // first slot ever pushed
  float4 *d_sparse = nullptr;        // sparse convolution: kept taps per anchor and link (ring)
  int32_t *d_sparse_dly = nullptr;
  uint64_t sparse_bytes = 0;
  // what each lane's device cursor holds for this UE (after queued work); UINT64_MAX: unknown
  uint64_t dev_cursor[tt_engine::kLanes] = {UINT64_MAX, UINT64_MAX, UINT64_MAX, UINT64_MAX,
                                            UINT64_MAX, UINT64_MAX, UINT64_MAX, UINT64_MAX};
  std::deque<std::pair<uint64_t, uint64_t>> inflight;  // (slot_end, batch seq)
  std::deque<std::pair<uint64_t, int64_t>> arrivals;   // served requests not launched yet: (slot, arrival ns)
  bool in_pending = false;                             // listed in the engine's pending list
  tt_cell *cell = nullptr;      // uplink aggregation cell consuming this channel's outputs
  // sum-of-sinusoids synthesis: the trace is a ring of anchors refilled before each run
  bool synth = false;
  float *d_amp = nullptr;
  double *d_freq = nullptr, *d_phase = nullptr;
  int synth_m = 0;
  double synth_fs = 0.0;
  // timed trace (entries every src_step samples): d_taps is a ring of anchors refilled before each
  // run by FP64 trace-time interpolation from the stored trace d_src
  bool retime = false;
  float2 *d_src = nullptr;
  uint64_t src_T = 0;
  double src_step = 0.0;
  int src_loop = 0;
};

struct tt_cell {
  tt_engine *e = nullptr;
  tt_cell_config cfg{};
  int n = 0, Q = 0;
  size_t slot_out_elems = 0;    // int16 values per slot
  int16_t *d_out = nullptr;
  uint64_t ring_bytes = 0;
  std::vector<tt_chan *> members;
  TTCellMember *d_members = nullptr;
  size_t members_cap = 0;
  bool started = false;
  uint64_t launched_end = 0, completed_end = 0, pulled_end = 0;
  std::deque<std::pair<uint64_t, uint64_t>> inflight;  // (slot_end, batch seq)
};


// Return TT_ERR_CUDA with the failing call and CUDA's message (inside a function returning tt_status).
#define TT_CK(call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return ttx::fail(TT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

namespace ttx {

// Device memory of the engine: through the allocator hook if one is set, else cudaMalloc/cudaFree.
// dev_free waits for the engine's streams first (cudaFree's implicit synchronisation, kept for
// the hook) and ignores null.
cudaError_t dev_alloc(tt_engine *e, void **p, size_t bytes);
void dev_free(tt_engine *e, void *p);
template <class T>
cudaError_t dmalloc(tt_engine *e, T **p, size_t bytes) {
  return dev_alloc(e, reinterpret_cast<void **>(p), bytes);
}
inline void dfree(tt_engine *e, void *p) { dev_free(e, p); }

// NVTX range for the duration of a scope (names the engine's calls in a profiler's timeline).
struct NvtxScope {
  explicit NvtxScope(const char *name);
  ~NvtxScope();
};

// Record a message for tt_last_error() and return the status.
tt_status fail(tt_status s, const char *fmt, ...);
int64_t now_us();
int64_t now_ns();
cudaEvent_t get_event(tt_engine *e);
// Poll batch events in order (engine lock held); returns the first hard CUDA error seen.
cudaError_t update_completed(tt_engine *e);
void update_chan(tt_chan *c);
// TT_OK if slots [first, first + n) may be pushed now (engine lock held).
tt_status check_room(tt_chan *c, uint64_t first, uint32_t n);
void mark_pushed(tt_chan *c, uint64_t first, uint32_t n);                      // arrival: now
void mark_pushed_at(tt_chan *c, uint64_t first, uint32_t n, int64_t arrival_ns);
// Wait (bounded) until batch `seq` is complete (engine lock held, released while blocking).
tt_status wait_seq(tt_engine *e, uint64_t seq, int64_t timeout_us, std::unique_lock<std::mutex> &lk);
// Copy slots [first, first + n) between a linear buffer and a ring of Q slots (at most 2 copies).
cudaError_t ring_copy(int16_t *ring, size_t slot_elems, int Q, uint64_t first, uint32_t n, const void *src, void *dst,
                      cudaMemcpyKind kind, cudaStream_t st, bool to_ring);

// Tiled-kernel geometry helpers (tt_engine.cpp): chunk table of a channel, delay class, switch
// of a channel's geometry, sparse convolution on, handle validity.
std::vector<int32_t> chunk_table(const std::vector<uint32_t> &L, int spt, int tpb, int *max_touched);
int pick_dclass(int d_max);
tt_status set_geom(tt_chan *c, int spt, int tpb);
bool sparse(const tt_chan *c);
bool valid_chan(const tt_chan *c);

// ---- traces and the per-run anchor pre-passes (tt_traces.cpp; engine lock held) ----
tt_status launch_retime(tt_engine *e, const std::vector<tt_chan *> &chans);
tt_status launch_synth(tt_engine *e, const std::vector<tt_chan *> &chans);
tt_status launch_topn(tt_engine *e, const std::vector<tt_chan *> &chans);

// ---- uplink cells (tt_cells.cpp) ----
// Engine lock held: an uplink cell has member slots to aggregate and ring room for them.
bool cells_have_work(const tt_engine *e);
// Engine lock held: aggregate every slot all members of each cell have launched (after their
// kernels, on the engine stream); ends receives (cell, new launched end) per launched cell.
tt_status launch_cells(tt_engine *e, std::vector<std::pair<tt_cell *, uint64_t>> &ends);

// ---- serving hooks (tt_server.cpp) ----
// A push of [first, first + n) became visible (engine lock held): its arrival is recorded.
void server_note_push(tt_chan *c, uint64_t first, uint32_t n, int64_t arrival_ns);
// Batch `seq` launched channel c's slots [from, to) (engine lock held).
void server_note_launch(tt_chan *c, uint64_t from, uint64_t to, uint64_t seq);
// Before a batch's completion event: stamp its completion on the device, on stream st (engine lock held).
tt_status server_stamp(tt_engine *e, uint64_t seq, cudaStream_t st);
// Before a batch's first kernel: stamp when the device starts it, on stream st (engine lock held).
tt_status server_stamp_start(tt_engine *e, uint64_t seq, cudaStream_t st);
// Create launch lanes up to n (at most tt_engine::kLanes; engine lock held); false leaves the engine
// on the lanes it had.
bool enable_lanes(tt_engine *e, int n);
// Wait for every stream of the engine (all lanes, copies).
void sync_all(tt_engine *e);
// A push found the ring full while a server runs: wait (engine lock held, released while waiting)
// until room() or the queue timeout; TT_OK or the failure status.
template <class Room>
tt_status server_wait_room(tt_engine *e, std::unique_lock<std::mutex> &lk, Room room);
// A push waited for ring room (refused: the wait ran out); counted in the server's report.
void server_count_wait(tt_engine *e, bool refused);
// A channel was destroyed: admission waiters may now fit.
void admission_notify(tt_engine *e);
// The thread running the server's batching loop (tt_engine_run from others is refused).
bool is_server_thread(const tt_engine *e);
int64_t server_queue_timeout_us(const tt_engine *e);

// ---- tiled-kernel geometry and the autotuner (tt_engine.cpp, tt_tune.cpp) ----
// Samples-per-thread values a channel's symbol lengths allow, largest first, none above cap.
std::vector<int> spt_candidates(const std::vector<uint32_t> &L, uint32_t cap, uint32_t n_rx, uint32_t n_tx);
// Shared memory of a traced channel at (spt, tpb); 0 if it does not fit (engine lock held).
size_t smem_need(const tt_chan *c, int spt, int tpb, int *tap_need);
// Switch a traced channel to (spt, tpb) (engine lock held); upload_desc publishes it.
tt_status apply_geom(tt_chan *c, int spt, int tpb);
tt_status upload_desc(tt_chan *c);
void drop_graph(tt_engine *e);
// One batched launch of slots [first[i], first[i] + count[i]) of chans[i], as a run launches it:
// a warm-up, then the best of reps timings between events a and b (engine lock held).
tt_status time_batch(tt_engine *e, const std::vector<tt_chan *> &chans, const std::vector<uint64_t> &first,
                     const std::vector<uint64_t> &count, int reps, cudaEvent_t a, cudaEvent_t b, float *best_ms);
// Tuning class of an FP32 channel with this trace: symbol lengths, antennas, tap-count bucket (next
// power of two, at least 8), delay class, AWGN on/off, output format, top-n.
std::string tune_class_key(const tt_chan *c, uint32_t n_taps, int dclass);
// Samples-per-thread cap of the autotuner's search (the engine's setting, else 16).
uint32_t tune_spt_cap(const tt_engine *e);
// The cached choice for a class on this engine's device model (any thread).
bool tune_lookup(tt_engine *e, const std::string &key, int *spt, int *tpb);
// Read TT_TUNE_CACHE (if set) into the engine's cache; a missing file is an empty cache.
void tune_load(tt_engine *e);

template <class Room>
tt_status server_wait_room(tt_engine *e, std::unique_lock<std::mutex> &lk, Room room) {
  const int64_t deadline = now_us() + server_queue_timeout_us(e);
  bool counted = false;
  for (;;) {
    tt_status st = room();
    if (st != TT_ERR_AGAIN || !e->server) return st;
    if (!counted) {
      server_count_wait(e, false);
      counted = true;
    }
    const int64_t left = deadline - now_us();
    if (left <= 0) {
      server_count_wait(e, true);
      return st;
    }
    e->room_cv.wait_for(lk, std::chrono::microseconds(left < 1000 ? left : 1000));
  }
}

}  // namespace ttx
