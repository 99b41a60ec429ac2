/*
 * tt_chan.h -- C ABI of the GB300 per-UE channel-convolution engine.
 *
 * The operation (paper Sec. III-B): every UE u gets its own linear,
 * time-varying convolution of the transmitted complex baseband IQ stream,
 *     y_u(t) = x(t) * h_u(t),
 * with h_u read from a channel trace of discrete complex taps on a fixed
 * delay grid per time step (Sec. IV, "Tiny-Twin compatible channel traces"),
 * convolution kept per UE so that UEs are isolated from one another
 * (Sec. III-C, "Parallelizing Convolution Computation").  In sample form, for
 * Rx antenna r and absolute sample index m:
 *
 *     y_r[m] = sum_t sum_k h_{r,t,k}(m) * x_t[m - d_k] + w_r[m]
 *
 *   h(m)  = H[a] + ((m - b_a) / L_a) * (H[a+1] - H[a])   for b_a <= m < b_a + L_a,
 *           a = absolute OFDM symbol index, b_a its first sample, L_a its length;
 *   H[a]  = the trace entry of symbol a (step_samples == 0), or the FP64 linear
 *           interpolation of the trace in time at sample b_a (step_samples > 0);
 *   d_k   = integer sample delays shared by all antenna pairs of a UE;
 *   x_t[m] = 0 before the first slot a UE ever processes (empty delay line);
 *   w_r[m] = optional AWGN, variance noise_var per complex sample, from
 *           Philox4x32-10 (key = seed, counter = (m>>1, ue_id, r)) and Box-Muller;
 *   output = clamp(round_half_even(y), -32768, 32767) per I and Q.
 *
 * Units.  A slot is samples_per_slot complex samples per antenna, split into
 * symbols_per_slot OFDM symbols.  IQ buffers are int16, I and Q interleaved,
 * laid out [antenna][sample][2]: a slot of input is n_tx*N*2 int16 values,
 * a slot of output n_rx*N*2 (or n_rx*N complex64 with TT_OUT_CF32).
 * Several consecutive slots are laid out slot-major: [slot][antenna][sample][2].
 *
 * Ownership.  The library owns every device allocation it makes.  Caller
 * buffers (host or device) are borrowed only for the duration of the call,
 * except where a function says it works asynchronously on the caller's stream.
 * Handles are not thread-safe individually: use one tt_chan from one thread
 * at a time, with one exception: one producer thread may push to a channel
 * (tt_chan_push_slot(s)) while one consumer thread pulls from it
 * (tt_chan_pull_slot(s)).  An engine serialises its own state, so different
 * channels of one engine may be used from different threads; push and pull
 * wait for their copies with the engine unlocked, so host-to-device and
 * device-to-host copies of different threads overlap.
 *
 * Errors.  Every function returns a tt_status.  On error no out-parameter is
 * written, and tt_last_error() returns a thread-local message.  There is no CPU
 * fallback: without a usable CUDA device tt_engine_create fails with
 * TT_ERR_CUDA.
 */
#ifndef TT_CHAN_H
#define TT_CHAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_CHAN_ABI_VERSION 4

typedef struct tt_engine tt_engine; /* one per GPU: stream, HBM budget, form, UE table */
typedef struct tt_chan tt_chan;     /* one per UE link: config, trace, delay line, rings */

typedef int32_t tt_status;
enum {
  TT_OK = 0,
  TT_ERR_INVALID = -1,   /* bad argument, size or layout */
  TT_ERR_NO_MEMORY = -2, /* admission refused by the HBM budget, or an allocation failed */
  TT_ERR_CUDA = -3,      /* CUDA runtime failure (no device, launch error, ...) */
  TT_ERR_TRACE = -4,     /* malformed trace: sizes, delays out of range, non-finite taps */
  TT_ERR_AGAIN = -5,     /* nothing ready yet, or the slot ring is full */
  TT_ERR_TIMEOUT = -6,   /* a bounded wait ran out */
  TT_ERR_STATE = -7,     /* out-of-order slot, no trace loaded, wrong form, bad state blob */
  TT_ERR_IO = -8         /* the tuning cache file (TT_TUNE_CACHE) could not be written */
};

/* How tt_engine_run executes pending slots. */
enum {
  TT_FORM_BATCHED = 0, /* one tiled kernel over every pending (UE, slot) of all UEs */
  TT_FORM_PLAIN = 1    /* comparison form: one simple launch per UE per slot */
};

/* Arithmetic of a channel. TT_FP32 is the reference-accuracy CUDA-core path. */
enum { TT_FP32 = 0, TT_BF16_TC = 1, TT_FP16_TC = 2 };

/* Output sample format.  TT_OUT_CF32 skips the int16 packing and returns y
 * itself as complex64 (re, im float32): output buffers are then
 * [n_rx][N] x 8 bytes per slot instead of [n_rx][N][2] int16. */
enum { TT_OUT_INT16 = 0, TT_OUT_CF32 = 1 };

typedef struct {
  uint32_t struct_size;      /* sizeof(tt_engine_config) */
  int32_t device;            /* CUDA device ordinal */
  uint64_t hbm_budget_bytes; /* admission limit for all channels; 0 = no limit */
  uint32_t form;             /* TT_FORM_* */
  uint32_t max_ues;          /* capacity of the device UE table; 0 = 1024 */
  uint32_t samples_per_thread; /* cap on the tiled kernel's samples per thread: 0 = 8 (more, shorter
                                  work items: the latency setting); else 1, 2, 4, 8 or 16 (16 only for
                                  channels with at most 2 Rx antennas; it runs bulk single-antenna
                                  work faster).  Each channel uses the largest allowed value dividing
                                  all its symbol lengths. */
  uint32_t threads_per_block;  /* tiled kernel's threads per CTA: 0 = 128 unless the tuning cache or
                                  tt_engine_autotune picks 256 for a channel's class; 128 or 256 =
                                  every channel uses it (the tuner then searches samples per thread
                                  only, and cached choices of the other count are ignored) */
  uint32_t persistent;       /* 1: persistent CTAs claim work items from a device counter; 0: by stride */
  uint32_t graphs;           /* 1: tt_engine_run captures its launches in a CUDA graph and replays it
                                while the set of channels and slots per run stays the same;
                                consecutive replays rotate over four launch lanes (each with its own
                                graph instance), so they overlap on the GPU (not with uplink cells) */
  /* Optional allocator hook (both set, or both NULL for cudaMalloc/cudaFree).  Every device buffer
   * the engine owns (rings, traces, tables, work lists) comes from dev_alloc(bytes, alloc_ctx), which
   * returns device memory on cfg->device aligned to 256 bytes, or NULL (then the call fails with
   * TT_ERR_NO_MEMORY or TT_ERR_CUDA).  The engine calls dev_free(ptr, alloc_ctx) only after its own
   * streams are idle, so the allocator may hand the memory to other work at once.  The hooks may
   * be called from any engine call and from the serving thread (tt_server_start).  Fields present
   * when struct_size covers them. */
  void *(*dev_alloc)(size_t bytes, void *ctx);
  void (*dev_free)(void *ptr, void *ctx);
  void *alloc_ctx;
} tt_engine_config;

typedef struct {
  uint32_t struct_size;       /* sizeof(tt_chan_config) */
  uint32_t ue_id;             /* keys the AWGN stream; need not be unique */
  uint32_t samples_per_slot;  /* N, 1 .. 2^24 */
  uint32_t symbols_per_slot;  /* 1 .. 32 (14 for NR) */
  const uint32_t *symbol_len; /* [symbols_per_slot], summing to N; copied */
  uint32_t n_tx, n_rx;        /* 1 .. 4 each */
  uint32_t max_taps;          /* upper bound on the trace's tap count, 1 .. 128 */
  uint32_t max_delay;         /* upper bound on the delays, samples, <= 1024 */
  uint32_t ring_slots;        /* slot ring depth Q (>= 2 + ceil(max_delay/N)); 0 = that minimum + 2 */
  uint64_t seed;              /* AWGN key */
  float noise_var;            /* sigma^2 per complex sample; 0 disables AWGN */
  uint32_t precision;         /* TT_FP32: CUDA-core FP32 path.  TT_BF16_TC / TT_FP16_TC: block-Toeplitz
                                 tensor-core path (tcgen05, FP32 accumulation), delays <= 127 */
  uint32_t output_format;     /* TT_OUT_INT16 (packed IQ) or TT_OUT_CF32 (complex64 before packing) */
  uint32_t top_n;             /* sparse convolution (Sec. III-C): 0 = every tap; n > 0 = for each OFDM
                                 symbol and (r, t) link only the n taps of largest |H[a]|^2 at the
                                 symbol's anchor a (ties: lower tap index), each interpolated toward
                                 its H[a+1].  The kernel ranks binary32 powers p = fma(re, re, im * im),
                                 so where two powers lie within binary32 rounding of each other at the
                                 n-th place, either tap may be the one kept.
                                 TT_FP32 batched form only (TT_ERR_INVALID otherwise) */
} tt_chan_config;

typedef struct {
  uint32_t struct_size;    /* sizeof(tt_trace_desc) */
  const float *taps;       /* complex64, re/im interleaved, [n_anchors][n_rx][n_tx][n_taps]; copied */
  const int32_t *delays;   /* [n_taps], non-decreasing, 0 <= d <= max_delay; copied */
  uint32_t n_anchors;      /* >= 1 */
  uint32_t n_taps;         /* 1 .. max_taps */
  double step_samples;     /* 0: one trace entry per OFDM symbol; > 0: entry i sits at sample i*step */
  int32_t loop;            /* 1: the trace wraps around; 0: it holds its last entry */
} tt_trace_desc;

typedef struct {
  uint64_t hbm_in_use;      /* bytes allocated for admitted channels */
  uint64_t hbm_budget;      /* the admission limit (0 = none) */
  uint32_t n_chans;         /* admitted channels */
  uint32_t pad;
  uint64_t launches;        /* kernel launches issued by tt_engine_run so far */
  uint64_t slots_processed; /* (UE, slot) pairs launched so far */
  uint64_t graph_builds;    /* CUDA graphs captured (graphs mode) */
  uint64_t graph_launches;  /* CUDA graph replays (graphs mode) */
} tt_engine_stats;

/* ---------------------------------------------------------------- engine */

/* Create an engine on cfg->device.  Fails with TT_ERR_CUDA if there is no
 * such device.  *out receives the handle. */
tt_status tt_engine_create(const tt_engine_config *cfg, tt_engine **out);

/* Wait for all work, then free everything, including channels not yet destroyed. */
tt_status tt_engine_destroy(tt_engine *e);

/* Launch every pushed-but-not-launched slot of every channel (in push order
 * per channel).  Asynchronous: returns once the work is queued on the
 * engine's stream.  Channels without a trace are skipped. */
tt_status tt_engine_run(tt_engine *e);
/* The slot-synchronous name of tt_engine_run: one launch (or graph replay) for every pushed slot. */
tt_status tt_engine_run_slot(tt_engine *e);

/* Slot-synchronous replay: n_steps times, every started, traced channel
 * releases its launched outputs, commits its next slots_per_step slots in
 * place (the input ring already holds their IQ: whatever the caller last
 * wrote at those ring positions) and tt_engine_run launches them all.
 * Asynchronous like tt_engine_run.  TT_ERR_AGAIN if a ring has no room. */
tt_status tt_engine_replay(tt_engine *e, uint32_t n_steps, uint32_t slots_per_step);

/* Make the engine's stream (tt_engine_stream) wait, on the device, for every batch launched so
 * far, whichever launch lane it runs on, so that work or a CUDA event queued on that stream
 * afterwards follows all of them (for example the end event when timing a series of runs: batches
 * of a graph-replaying or serving engine run on several lanes).  Does not block the host. */
tt_status tt_engine_join(tt_engine *e);

/* Block until all launched work is complete, at most timeout_us (< 0: no limit).
 * TT_ERR_TIMEOUT if it is still running, or if a tensor-core kernel reported
 * that one of its bounded waits expired (the affected slots are invalid). */
tt_status tt_engine_sync(tt_engine *e, int64_t timeout_us);

/* Bounds-checked build.  The library can be built a second time with
 * TT_CHECKED=1 (libttchan_checked.so beside libttchan.so; the Python binding
 * loads it when the environment variable TT_CHECKED is 1).  There the tiled
 * FP32 kernel and the tensor-core kernel test every shared-, tensor- and
 * global-memory index before the access.
 * An index out of bounds is not accessed: the kernel counts it in the
 * engine's check report and keeps the code of the first one, without a trap,
 * so the GPU and the process stay usable (the affected slots' outputs are
 * invalid).  Codes: 1 staged input window (shared) written, 2 input ring
 * read, 3 tap buffer (shared), 4 trace or sparse tap ring read, 5 delay
 * buffer (shared), 6 symbol table (shared), 7 phase planes (shared) written,
 * 8 staged input window read, 9 phase planes read, 10 tap or delay buffer
 * read by the tap loop, 11 output ring written, 12 tensor-memory column
 * (tensor-core kernel; there codes 1 and 3 also cover its staged signal and
 * tap tables).  tt_engine_get_check waits for the launched work, reads the
 * report and clears it.  In the normal build checked_build is 0 and the
 * report stays empty.  The static entry (tt_conv_static) and the auxiliary
 * passes (synthesis, retiming, top-n selection, cells) are not instrumented. */
typedef struct {
  uint32_t checked_build; /* 1: this library tests indices */
  uint32_t violations;    /* out-of-bounds indices since the last call (not accessed) */
  uint32_t first_code;    /* the first one's code (list above), 0 if none */
  uint32_t pad;
} tt_check_report;
tt_status tt_engine_get_check(tt_engine *e, tt_check_report *out);

/* The engine's CUDA stream (a cudaStream_t) for ordering caller work. */
tt_status tt_engine_stream(tt_engine *e, void **stream);

tt_status tt_engine_get_stats(tt_engine *e, tt_engine_stats *out);

/* Autotune the tiled FP32 kernel's geometry for every class of admitted,
 * traced FP32 channels (same symbol lengths, antennas, tap-count bucket: the
 * next power of two, at least 8, delay class, AWGN on/off, output format,
 * top-n).  Two axes: samples per thread
 * S in {1, 2, 4, 8, 16} (those dividing every symbol length, 16 with at most
 * 2 Rx antennas, none above the engine's samples_per_thread setting or 16
 * when it is 0) and threads per CTA in {128, 256}; a work item (the tile)
 * spans S x threads samples, 128 to 4096.  The objective is the whole batch:
 * one slot of every channel that has a free ring position (written to that
 * free position, so no queued or unpulled slot is touched), launched as
 * tt_engine_run launches it, best of `reps` timings.  Classes are visited
 * largest first; each (S, threads) pair that fits shared memory replaces the
 * class's current choice only if the batch gets at least 1% faster in two
 * timings in a row.  Waits
 * for queued work first.  *classes_tuned (may be NULL) receives the number of
 * classes that had a choice to make.
 *
 * Tuning cache: if the environment variable TT_TUNE_CACHE names a file when
 * the engine is created, the engine reads the choices stored there for its
 * device model (device name and SM count); a channel of a stored class starts
 * at the stored geometry when its trace is loaded.  tt_engine_autotune writes
 * every class's choice back into that file (lines of other device models and
 * classes are kept; the file is replaced through a temporary file and a
 * rename).  TT_ERR_IO if it cannot be written; the tuned geometry stays in
 * effect for the engine.  Unreadable or malformed lines are ignored. */
tt_status tt_engine_autotune(tt_engine *e, int32_t reps, uint32_t *classes_tuned);

/* The work decomposition a channel launches with (for reports and tests). */
typedef struct {
  uint32_t tensor_core;        /* 1: tensor-core kernel (BF16/FP16 precision), 0: tiled FP32 kernel */
  uint32_t samples_per_thread; /* tiled kernel: S (0 for the tensor-core kernel) */
  uint32_t threads_per_cta;    /* tiled kernel: 128 or 256 (0 for the tensor-core kernel) */
  uint32_t samples_per_item;   /* tiled kernel: the tile, S x threads_per_cta */
  uint32_t items_per_slot;     /* work items (CTAs' units of work) per slot */
  uint32_t has_trace;          /* 0: the geometry is provisional until a trace is loaded */
} tt_chan_geometry;
tt_status tt_chan_get_geometry(tt_chan *c, tt_chan_geometry *out);

/* Serving benchmark.  Generates requests on the calling thread for warmup_s +
 * duration_s seconds: every channel with a trace receives slot-push requests
 * at Poisson times (mean inter-arrival slot_period_us, plus uniform
 * +-jitter_us, kept increasing).  A request commits the UE's next slot in
 * place: the IQ the caller left at that ring position (device-resident input).
 * The requests go through the serving path of tt_server_start (started and
 * stopped by this call): its batching thread launches them, and their latency
 * is the device-stamped completion of their batch minus their arrival.  A
 * request that finds the UE's ring full waits in a per-UE queue of 64 and is
 * committed, with its own arrival time, when completed slots free the ring;
 * only a request that finds that queue full is refused.  Latencies count the
 * requests that arrived after the warm-up.
 * release_outputs = 1 frees each output ring position as soon as it is
 * complete, the rings of uplink aggregation cells included; 0 keeps the
 * outputs for tt_chan_pull_* / tt_cell_pull_slots (rings then fill up). */
typedef struct {
  uint32_t struct_size;           /* sizeof(tt_serve_config) */
  uint32_t max_slots_per_ue;      /* 0 = no limit; else each UE stops after this many requests */
  double warmup_s, duration_s;    /* arrivals before the measured window, and its length */
  double slot_period_us;          /* mean inter-arrival per UE (500 = one 30 kHz slot) */
  double jitter_us;               /* uniform +- jitter added to each inter-arrival */
  double deadline_us;             /* latency bound counted as a miss (0 = 500) */
  uint64_t seed;                  /* arrival-process seed */
  uint32_t release_outputs;
  uint32_t max_inflight_batches;  /* as tt_server_config (0 = 8) */
} tt_serve_config;

typedef struct {
  uint64_t requests, refused, completed, batches, deadline_misses;
  double mean_batch;              /* requests per batch */
  double throughput;              /* completed requests (UE-slots) per second of the measured window */
  double p50_us, p99_us, p999_us, max_us, mean_us;  /* device-stamped completion - arrival */
  double stamp_error_us, gpu_us_per_batch, gpu_busy; /* as tt_server_report */
} tt_serve_report;

tt_status tt_engine_serve(tt_engine *e, const tt_serve_config *cfg, tt_serve_report *out);

/* Serving with callers' own pushes: continuous batching of slot pushes from many UEs as they
 * arrive, each UE isolated from the others (Sec. III-C).  tt_server_start starts an engine-owned batching
 * thread.  From then on every slot pushed by any thread, through tt_chan_push_slot(s)(_dev),
 * tt_engine_push_slots or tt_chan_commit_slots, is a request.  Its arrival time is the push call's
 * host steady-clock time.  The thread launches whatever is pending as one batch whenever fewer
 * than max_inflight_batches run, so requests that arrive while others are on the GPU join the
 * next batch.  tt_engine_run from any other thread returns TT_ERR_STATE meanwhile.
 *
 * Back-pressure is a queue, not a refusal: a push that finds its slot ring full waits (the calling
 * thread blocks) until completed, released outputs free room, for up to queue_timeout_us.  Only
 * then does it return TT_ERR_AGAIN (counted as refused).
 *
 * Each batch's completion is stamped on the device: a one-thread kernel after the batch's kernels
 * writes %globaltimer into pinned host memory.  tt_server_start calibrates that clock against the
 * host steady clock (the shortest of 32 launch round trips, uncertainty = half of it).  A request's
 * latency is its batch's device stamp, on the host clock, minus its arrival.  tt_server_stop waits
 * for every launched batch, stops the thread and fills the report.  The batching thread polls the
 * running batch without the engine lock, so pushing threads are not kept waiting by it. */
typedef struct {
  uint32_t struct_size;           /* sizeof(tt_server_config) */
  uint32_t max_inflight_batches;  /* 0 = 8; each batch in flight gets its own launch lane (streams,
                                     work list, counters), so consecutive batches overlap on the GPU
                                     (not while the engine has uplink cells) */
  uint32_t release_outputs;       /* 1: completed slots' outputs are released without pulls */
  int32_t queue_timeout_us;       /* wait of a push into a full ring: 0 = 1 s, < 0 = no wait */
  double deadline_us;             /* latency counted as a deadline miss above this (0 = 500) */
  double warmup_us;               /* requests arriving earlier after the start are not counted */
  double coalesce_us;             /* while a batch runs, the next one forms until its oldest request
                                     has waited this long (0 = 20); with none running it launches at once */
} tt_server_config;

typedef struct {
  uint32_t struct_size;           /* sizeof(tt_server_report) */
  uint64_t requests;              /* slots pushed while serving (warm-up included) */
  uint64_t completed;             /* requests after the warm-up whose latency was measured */
  uint64_t queued;                /* pushes that found the ring full and waited for room */
  uint64_t refused;               /* pushes whose wait ran out (TT_ERR_AGAIN) */
  uint64_t batches, deadline_misses;
  double mean_batch;              /* requests per batch */
  double p50_us, p99_us, p999_us, max_us, mean_us, min_us;
  double stamp_error_us;          /* uncertainty of the device-clock calibration */
  double gpu_us_per_batch;        /* device time from a batch's first kernel to its completion stamp */
  double gpu_busy;                /* those times' sum over the span from the first start to the last end */
} tt_server_report;

tt_status tt_server_start(tt_engine *e, const tt_server_config *cfg);
tt_status tt_server_stop(tt_engine *e, tt_server_report *out);

/* Admission with a waiting list: like tt_chan_create, but a channel that does not fit the HBM
 * budget waits (the calling thread blocks) until channels destroyed on this engine free enough
 * memory, or for timeout_us (< 0: no limit).  Waiters are admitted in arrival order: a later
 * request does not overtake an earlier one that still waits.  TT_ERR_NO_MEMORY when the wait runs
 * out; other errors as tt_chan_create. */
tt_status tt_chan_create_queued(tt_engine *e, const tt_chan_config *cfg, int64_t timeout_us, tt_chan **out);

/* ---------------------------------------------------------------- channel */

/* Admit a channel: allocates its slot rings if they fit in the budget
 * (TT_ERR_NO_MEMORY otherwise).  The delay line starts empty (zeros). */
tt_status tt_chan_create(tt_engine *e, const tt_chan_config *cfg, tt_chan **out);

/* Free the channel's device memory (after its launched work completes). */
tt_status tt_chan_destroy(tt_chan *c);

/* Copy a trace to the device (replacing any previous one).  Counted against
 * the budget: TT_ERR_NO_MEMORY if it does not fit, TT_ERR_TRACE if malformed.
 * A trace with step_samples > 0 also takes a ring of (ring_slots + 1) x
 * symbols_per_slot + 1 per-symbol anchors, which each tt_engine_run refills
 * (FP64 trace-time interpolation) for the slots it launches; it is counted too.
 * Not allowed while the channel has launched work in flight (TT_ERR_STATE). */
tt_status tt_chan_load_trace(tt_chan *c, const tt_trace_desc *trace);

/* A continuous CIR: per time step, n_paths paths with complex gains per
 * (r, t) link and delays in samples (delay x sampling rate, any real >= 0). */
typedef struct {
  uint32_t struct_size;       /* sizeof(tt_cir_desc) */
  uint32_t n_steps, n_paths;  /* time steps (the trace's anchors) and paths per step */
  uint32_t n_taps;            /* delay grid 0 .. n_taps-1 (<= max_taps, n_taps-1 <= max_delay) */
  const float *gains;         /* complex64 [n_steps][n_rx][n_tx][n_paths] */
  const double *delays;       /* [n_steps][n_paths], samples */
  double step_samples;        /* as tt_trace_desc: 0 = one step per OFDM symbol */
  int32_t loop;               /* as tt_trace_desc */
  uint32_t reserved;
} tt_cir_desc;

/* Trace ingestion (Sec. IV: a continuous CIR is resampled onto a fixed delay
 * grid for each time step, the method unnamed).  The device computes, in FP64,
 *   H[t][r][x][k] = sum_p gains[t][r][x][p] * sinc(k - delays[t][p]),
 *   sinc(v) = sin(pi v) / (pi v),  k = 0 .. n_taps-1,
 * the band-limited discrete-time equivalent of the multipath channel, rounds
 * it to complex64 and installs it as the channel's trace with delays 0 ..
 * n_taps-1, exactly as tt_chan_load_trace would; paths outside the grid
 * leave sinc tails inside it.  Errors as tt_chan_load_trace; TT_ERR_TRACE for
 * a non-finite gain or a negative or non-finite delay. */
tt_status tt_chan_load_cir(tt_chan *c, const tt_cir_desc *cir);

/* Sum-of-sinusoids tap processes synthesised on the device (Sec. IV: 3GPP
 * traces whose time variation comes from a Jakes-based Doppler model).  Tap
 * (r, x, k) at anchor a, which sits at t = b_a / sample_rate_hz seconds (b_a =
 * its first absolute sample), is
 *   amplitude[r][x][k] * M^(-1/2) * sum_n [cos(freq[..][n][0] t + phase[..][n][0])
 *                                     + j cos(freq[..][n][1] t + phase[..][n][1])]
 * (freq in rad/s; the Zheng-Xiao model is freq = w (cos a_n, sin a_n)).  The
 * phase is reduced modulo 2 pi in FP64, so long replays keep their accuracy;
 * the cosines and the sum are FP32.  The engine keeps a ring of anchors sized
 * for the channel's slot ring and fills each run's anchors before its
 * kernels, so no trace is stored: the channel replays indefinitely. */
typedef struct {
  uint32_t struct_size;       /* sizeof(tt_jakes_desc) */
  uint32_t n_taps;            /* K */
  uint32_t n_sinusoids;       /* M, 1 .. 64 */
  uint32_t reserved;
  const int32_t *delays;      /* [K], non-decreasing, <= max_delay */
  const float *amplitude;     /* [n_rx][n_tx][K] */
  const double *freq;         /* [n_rx][n_tx][K][M][2], rad/s */
  const double *phase;        /* [n_rx][n_tx][K][M][2], rad */
  double sample_rate_hz;      /* f_s > 0 */
} tt_jakes_desc;

tt_status tt_chan_load_jakes(tt_chan *c, const tt_jakes_desc *jakes);

/* Queue input slots [first, first+n).  The first push fixes the channel's
 * starting slot; after that slots must continue in order (TT_ERR_STATE).
 * TT_ERR_AGAIN if the ring has no room (pull or release outputs first).
 *   push_slots:     host buffer [n][n_tx][N][2], copied before return.
 *   push_slots_dev: device buffer, copied asynchronously after all work
 *                   previously queued on `stream` (a cudaStream_t, NULL = legacy
 *                   default stream); the buffer may be reused once that stream
 *                   has passed an event recorded after this call. */
tt_status tt_chan_push_slot(tt_chan *c, uint64_t slot, const int16_t *iq_in);
tt_status tt_chan_push_slots(tt_chan *c, uint64_t first, uint32_t n, const int16_t *iq_in);
tt_status tt_chan_push_slots_dev(tt_chan *c, uint64_t first, uint32_t n, const int16_t *d_iq_in,
                                 void *stream);
/* One slot from a device buffer [n_tx][N][2]: tt_chan_push_slots_dev with n = 1. */
tt_status tt_chan_push_slot_dev(tt_chan *c, uint64_t slot, const int16_t *d_iq_in, void *stream);

/* Zero-copy input: *d_ptr receives the device address inside the ring where
 * slot `slot`'s input ([n_tx][N][2]) lives.  Write it (on any stream, then
 * order that stream before the next tt_engine_run, e.g. by synchronising) and
 * commit it.  Valid for the next slot to push and the ring's free positions.
 * A position is free once the slot one ring depth earlier was pulled or
 * released.  tt_chan_release_slots needs only a launched slot, so after a
 * release ahead of completion, batches still running may read the position as
 * delay-line history: order the write after them too (tt_engine_sync, or the
 * engine stream after tt_engine_join).  The push calls order their copies
 * after such batches themselves. */
tt_status tt_chan_slot_input(tt_chan *c, uint64_t slot, int16_t **d_ptr);
tt_status tt_chan_commit_slots(tt_chan *c, uint64_t first, uint32_t n);

/* Pull the oldest not-yet-pulled slot into a host buffer [n_rx][N][2].
 * Waits at most timeout_us for it to complete (0: do not wait, < 0: no limit);
 * TT_ERR_AGAIN if it has not been launched (or nothing was pushed yet), TT_ERR_TIMEOUT if it is still
 * running. */
tt_status tt_chan_pull_slot(tt_chan *c, uint64_t *slot, void *iq_out, int64_t timeout_us);

/* Pull slots [first, first+n) (must be the oldest not yet pulled) into a host
 * buffer [n][n_rx][N][2], waiting as tt_chan_pull_slot does. */
tt_status tt_chan_pull_slots(tt_chan *c, uint64_t first, uint32_t n, void *iq_out,
                             int64_t timeout_us);

/* Device-side pull: copy slots [first, first+n) to a device buffer after
 * their computation; `stream` is made to wait for the copy.  Frees the ring
 * positions.  The slots must be launched already (TT_ERR_AGAIN otherwise). */
tt_status tt_chan_pull_slots_dev(tt_chan *c, uint64_t first, uint32_t n, void *d_iq_out,
                                 void *stream);
/* The oldest not-yet-pulled slot into a device buffer [n_rx][N][2], as tt_chan_pull_slots_dev
 * with n = 1; *slot receives its index (untouched on error). */
tt_status tt_chan_pull_slot_dev(tt_chan *c, uint64_t *slot, void *d_iq_out, void *stream);

/* Zero-copy output: device address of slot `slot`'s output ([n_rx][N][2]) in
 * the ring, valid until the slot is released.  Order reads after
 * tt_engine_sync or the engine stream.  Release frees ring positions of the
 * oldest not-yet-pulled slots. */
tt_status tt_chan_slot_output(tt_chan *c, uint64_t slot, const void **d_ptr);
tt_status tt_chan_release_slots(tt_chan *c, uint64_t first, uint32_t n);

/* Many channels in one call.  Entry i pushes slots [first[i], first[i]+n[i])
 * of chans[i] from the host buffer iq_in[i] (layout as tt_chan_push_slots),
 * or pulls them into iq_out[i] (layout as tt_chan_pull_slots).  Every entry is
 * checked before any copy starts (the first failing entry's status is
 * returned and nothing is copied); the copies are then queued back to back on
 * one copy stream and the call waits once, with the engine unlocked, for all
 * of them: per-channel calls would leave the copy engine idle between
 * channels.  Pull waits for the entries' slots to complete as
 * tt_chan_pull_slots does (timeout_us); a channel may appear at most once.
 * No counterpart in the paper, whose UE processes each move their own IQ. */
tt_status tt_engine_push_slots(tt_engine *e, uint32_t n_chans, tt_chan *const *chans, const uint64_t *first,
                               const uint32_t *n, const int16_t *const *iq_in);
tt_status tt_engine_pull_slots(tt_engine *e, uint32_t n_chans, tt_chan *const *chans, const uint64_t *first,
                               const uint32_t *n, void *const *iq_out, int64_t timeout_us);

/* ---- Uplink aggregation at a cell (Sec. III-A: the gNB convolves each UE's
 * uplink stream with that UE's channel and aggregates the results) ----
 * A cell owns an output ring of n_rx antennas.  Channels attached to it keep
 * running their own kernels; after them, every slot that all members have
 * launched is aggregated: the members' outputs summed in attach order (FP32),
 * plus the cell's AWGN (key (seed, cell_id), sigma^2 = noise_var), rounded and
 * saturated into the cell ring like a channel's output.  A member must have
 * the cell's samples_per_slot (even) and n_rx, TT_OUT_CF32 output, noise_var
 * 0, and no pushed slot yet; all members start at the same slot.  A member's
 * output slots are consumed by the aggregation (pulling or releasing them
 * gives TT_ERR_STATE).  If the cell ring is full the aggregation waits, the
 * members' rings fill, and pushes report TT_ERR_AGAIN until the cell is
 * pulled.  A member cannot be destroyed before its cell (TT_ERR_STATE).
 * No counterpart in the paper beyond the aggregation step itself. */
typedef struct tt_cell tt_cell;
typedef struct {
  uint32_t struct_size;       /* sizeof(tt_cell_config) */
  uint32_t cell_id;           /* keys the cell's AWGN stream */
  uint32_t samples_per_slot;  /* N of every member, even */
  uint32_t n_rx;              /* 1 .. 4, the Rx antennas of the cell and of every member */
  uint32_t ring_slots;        /* output ring depth, >= 1 (0 = 4) */
  uint32_t output_format;     /* TT_OUT_INT16 or TT_OUT_CF32 */
  uint64_t seed;              /* AWGN key */
  float noise_var;            /* sigma^2 per complex sample at the cell; 0 disables AWGN */
  uint32_t reserved;
} tt_cell_config;

tt_status tt_cell_create(tt_engine *e, const tt_cell_config *cfg, tt_cell **out);
tt_status tt_cell_attach(tt_cell *cell, tt_chan *c);
/* Pull cell slots [first, first+n) (the oldest not yet pulled) into a host
 * buffer [n][n_rx][N][2] (int16, or complex64 with TT_OUT_CF32), waiting as
 * tt_chan_pull_slots does; TT_ERR_AGAIN if they are not aggregated yet. */
tt_status tt_cell_pull_slots(tt_cell *cell, uint64_t first, uint32_t n, void *out, int64_t timeout_us);
/* Free the cell (after its queued work) and detach its members. */
tt_status tt_cell_destroy(tt_cell *cell);

/* Checkpoint / resume.  The state is the next slot index, the last
 * max_delay input samples per Tx antenna and the AWGN key; outputs that have
 * not been pulled are not part of it.  get_state with buf == NULL sets *len
 * to the size needed.  Both require no launched work in flight for this
 * channel (call tt_engine_sync first; TT_ERR_STATE otherwise).  After
 * set_state the next push must be the saved next slot; results are then
 * bit-identical to an uninterrupted run. */
tt_status tt_chan_get_state(const tt_chan *c, void *buf, size_t *len);
tt_status tt_chan_set_state(tt_chan *c, const void *buf, size_t len);

/* --------------------------------------------------- no-allocation entry point
 * The paper has no counterpart to this call.  It exists for callers that may
 * not allocate device memory: code inside another framework's memory pool or
 * a fixed-size real-time partition, or anything that must keep a constant
 * footprint.  tt_conv_static runs the same tiled kernel as tt_engine_run on
 * buffers the caller owns and calls no cudaMalloc, cudaFree or allocating
 * library routine.  Its scratch (descriptors, work list, chunk tables,
 * delays, work counters) lives in one fixed __device__ array inside the
 * library, about 200 KB, which every GPU that loads the library holds until
 * the process exits.
 *
 * Limits, rejected with TT_ERR_INVALID: at most 64 channels per call,
 * samples_per_slot <= 65536, at most 128 taps, delays <= 1024, and a
 * channel must fit the kernel's shared memory.  Alignment, also rejected with
 * TT_ERR_INVALID: d_ring_in 16-byte aligned, d_taps 8-byte, d_ring_out 4-byte
 * (TT_OUT_INT16) or 8-byte (TT_OUT_CF32).  Every argument is checked on the
 * host before the call touches the device.
 *
 * Layout and semantics follow the engine's rings: slot s of a channel sits at
 * ring position s % ring_slots, input [ring_slots][n_tx][N][2] int16, output
 * [ring_slots][n_rx][N] x (int16 I,Q | complex64).  The call computes slots
 * [first_slot, first_slot + n_slots) and reads the delay line from the ring
 * positions of earlier slots, so the caller keeps those filled (zeros before
 * the first slot).  Asynchronous on `stream` (cudaStream_t, NULL = legacy).
 *
 * The first call on a device looks up the scratch array's device address with
 * that device current.  Every call shares the array and leaves its contents behind; each call
 * rewrites what it reads and zeroes its counters.  Calls that overlap on the
 * GPU (different streams or threads) race on the array: order them on one
 * stream. */
typedef struct {
  uint32_t struct_size;       /* sizeof(tt_static_chan) */
  uint32_t ue_id;             /* keys the AWGN stream */
  uint32_t samples_per_slot;  /* N */
  uint32_t symbols_per_slot;
  const uint32_t *symbol_len; /* host, [symbols_per_slot], summing to N */
  uint32_t n_tx, n_rx;        /* 1 .. 4 */
  uint32_t ring_slots;        /* ring depth Q of both rings: >= n_slots + ceil(max delay / N), so that the
                                 delay line of the call's first slot is not overwritten by its own slots */
  const int16_t *d_ring_in;   /* device, caller-owned input ring */
  void *d_ring_out;           /* device, caller-owned output ring */
  const float *d_taps;        /* device, caller-owned complex64 [n_anchors][n_rx][n_tx][n_taps] */
  const int32_t *delays;      /* host, [n_taps], non-decreasing, 0 .. 1024 */
  uint32_t n_anchors, n_taps;
  double step_samples;        /* as in tt_trace_desc */
  int32_t loop;
  uint64_t seed;
  float noise_var;            /* sigma^2 per complex sample, 0 = off */
  uint32_t output_format;     /* TT_OUT_INT16 or TT_OUT_CF32 */
  uint64_t first_slot;        /* first slot to compute */
  uint32_t n_slots;           /* number of slots to compute */
} tt_static_chan;

tt_status tt_conv_static(const tt_static_chan *chans, uint32_t n_chans, void *stream);

/* ---------------------------------------------------------------- misc */

const char *tt_last_error(void);
int32_t tt_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TT_CHAN_H */
