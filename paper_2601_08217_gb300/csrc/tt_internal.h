// Internal types shared by the engine (host C++) and the CUDA kernels.
// Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#define TT_MAX_SYM 32
#define TT_MAX_ANT 4
#define TT_MAX_TAPS 128
#define TT_MAX_DELAY 1024
#define TT_TPB 128       // threads per CTA of the tiled kernel: the default choice
#define TT_TPB_WIDE 256  // the other choice the autotuner tries (a work item spans twice the samples)
#define TT_STATIC_MAX_CHANS 64            // channels per tt_conv_static call
#define TT_STATIC_MAX_ITEMS_PER_SLOT 512  // work items per slot in tt_conv_static (N <= 65536)

// Delay classes of the tiled kernel: the staged window is sized at compile
// time for delays up to these bounds.
#define TT_DCLASS0 128
#define TT_DCLASS1 256
#define TT_DCLASS2 512
#define TT_DCLASS3 1024

// Window geometry of the tiled kernel (TPB threads per CTA, samples per thread S, delay class
// DMAX): delay padding DP (a multiple of S) and phase-plane pitch NP in float2 words.
// NP is padded so that NP = 16/S (mod 16): sixteen consecutive window
// elements written by a half-warp then land in sixteen distinct 8-byte bank
// pairs (element e goes to plane e mod S, row e / S).
__host__ __device__ constexpr int tt_geo_dp(int S, int DMAX) { return (DMAX + S - 1) / S * S; }
__host__ __device__ constexpr int tt_geo_np_raw(int TPB, int S, int DMAX) {
  return (TPB * S + tt_geo_dp(S, DMAX)) / S + 1;
}
__host__ __device__ constexpr int tt_geo_np(int TPB, int S, int DMAX) {
  return tt_geo_np_raw(TPB, S, DMAX) + ((16 / (S < 16 ? S : 16)) % 16 - tt_geo_np_raw(TPB, S, DMAX) % 16 + 16) % 16;
}
__host__ __device__ constexpr int tt_dclass_max(int dclass) {
  return dclass == 0 ? TT_DCLASS0 : (dclass == 1 ? TT_DCLASS1 : (dclass == 2 ? TT_DCLASS2 : TT_DCLASS3));
}
// Longest input window of one work item (samples): the item's span plus the delay line.
__host__ __device__ constexpr int tt_geo_wmax(int TPB, int S, int DMAX) { return TPB * S + tt_geo_dp(S, DMAX); }

// Device-resident description of one admitted UE link.  The engine keeps an
// array of these on the device; work items index into it.
struct TTUEDesc {
  const int16_t *ring_in;  // [Q][n_tx][N][2]
  void *ring_out;          // [Q][n_rx][N] x (int16 I,Q | float2)
  const float2 *taps;      // [T][n_rx][n_tx][K]
  const int32_t *delays;   // [K]
  const int32_t *chunk_info;  // per work item of a slot: first symbol | (symbols touched << 16)
  const float4 *sparse;    // sparse convolution: [sparse_len][n_rx * n_tx][top_n] (H, dH) of the kept taps
  const int32_t *sparse_dly;  // and their delays; anchor a at a % sparse_len
  double step_samples;     // 0: one trace entry per symbol
  uint64_t seed;
  int32_t n;               // samples per slot
  int32_t nsym;            // symbols per slot
  int32_t n_tx, n_rx, n_taps;
  int32_t d_max;           // largest delay of the loaded trace
  int32_t top_n;           // 0: every tap; else the top_n taps per symbol and link (sparse convolution)
  int32_t sparse_len;      // anchors in the sparse ring
  int32_t ring_q;          // ring depth in slots
  int32_t n_anchors;
  int32_t loop;
  uint32_t ue_id;
  float noise_std;         // per I/Q component; 0 = AWGN off
  int32_t out_f32;         // 1: write y as float2 (no packing)
  int32_t spt;             // samples per thread of the tiled kernel for this UE
  int32_t dpad;            // d_max rounded up to a multiple of spt: delay-line part of the window
  int32_t groups;          // groups of spt samples per slot
  int32_t tpb;             // threads per CTA of the tiled kernel: groups per work item
  int32_t items_per_slot;  // CTAs (work items) per slot
  int32_t sym_start[TT_MAX_SYM + 1];  // symbol starts, sym_start[nsym] = n
  int32_t grp_start[TT_MAX_SYM + 1];  // first group of each symbol, grp_start[nsym] = groups
};

// A run of consecutive slots of one UE inside one launch.
struct TTSeg {
  uint64_t first_slot;
  uint32_t ue;          // index into the UE table
  uint32_t n_slots;
  uint32_t item_begin;  // first global work-item index of this run
  uint32_t items;       // n_slots * items_per_slot
};

// Bounds-checked build.  Compiled with -DTT_CHECKED=1 (a separate library), the tiled kernel and the
// tensor-core kernel test every shared-, tensor- and global-memory index before the access; an index out of bounds skips the access
// and is recorded here instead of faulting: report[0] counts violations, report[1] holds the code
// (TT_CHK_*) of the first.  In the normal build the tests compile away.
struct TTCheck {
  uint32_t *report;  // two words on the device, or null (violations are then skipped unrecorded)
  int32_t shrink;    // tests only: the output-store bound is lowered by this many words
  int32_t tap_max;   // set by the kernel: entries of each tap buffer
  int32_t kpad;      // set by the kernel: entries of each delay-offset buffer
};
enum {
  TT_CHK_RAW_WRITE = 1,   // staged raw window (shared), written by the copies
  TT_CHK_RING_IN = 2,     // input ring (global), read by the copies
  TT_CHK_TAP_SMEM = 3,    // tap buffer (shared)
  TT_CHK_TAP_GLOBAL = 4,  // trace or sparse tap ring (global)
  TT_CHK_DLY_SMEM = 5,    // delay-offset buffer (shared)
  TT_CHK_SYM = 6,         // symbol-start table (shared)
  TT_CHK_PLANE_WRITE = 7, // phase planes (shared), written by the conversion
  TT_CHK_RAW_READ = 8,    // staged raw window (shared), read by the conversion
  TT_CHK_PLANE_READ = 9,  // phase planes (shared), read by the tap loop
  TT_CHK_TAP_READ = 10,   // tap and delay-offset buffers (shared), read by the tap loop
  TT_CHK_RING_OUT = 11,   // output ring (global), written by the epilogue
  TT_CHK_TMEM = 12        // tensor memory column (tensor-core kernel)
};
int tt_checked_build();  // 1 in the TT_CHECKED library, else 0

struct TTLaunch {
  const TTUEDesc *ues;
  const TTSeg *segs;
  int n_segs;
  uint32_t total_items;
  uint32_t *counter;    // non-null: CTAs claim items from this device counter (zeroed before launch);
                        // null: CTA b takes items b, b + grid, b + 2 grid, ...
  int spt;              // 1, 2, 4, 8, 16
  int tpb;              // threads per CTA: TT_TPB or TT_TPB_WIDE (every UE of the launch has this)
  int nrx;              // 1..4 (every UE of the launch has this many Rx antennas)
  int ntx;              // 1..4 (every UE of the launch has this many Tx antennas)
  int dclass;           // delay class, see TT_DCLASS*
  int tap_max;          // largest (symbols touched x n_rx x n_tx x K) of the launch's UEs
  int k_max;            // largest tap count of the launch's UEs
  int grid;             // CTAs; < 0 on input asks for the occupancy (returned as -blocks per SM)
  size_t smem;          // dynamic shared memory bytes (tt_conv_smem_bytes)
  const unsigned long long *cursors;  // non-null: first slot of each run = cursors[ue] (graph replay)
  int topn;             // 1: every UE of the launch uses sparse convolution (top_n < its tap count)
  TTCheck check;        // bounds-checked build: where violations are recorded
};

// cursors[segs[i].ue] += segs[i].n_slots * stride for every segment (device-resident slot cursors).
cudaError_t tt_launch_advance(const TTSeg *segs, int n_segs, unsigned long long *cursors, unsigned stride,
                              cudaStream_t st);

// Dynamic shared memory of the tiled kernel for a launch.
size_t tt_conv_smem_bytes(int spt, int tpb, int dclass, int n_tx, int tap_max, int k_max);

// First symbol and number of symbols touched by each work item (tpb groups of spt samples) of a
// slot, packed jf | nst << 16; returns the item count, or -1 if it exceeds max_out.
int tt_conv_chunk_info(int spt, int tpb, const int32_t *sym_len, int nsym, int32_t *out, int max_out);
cudaError_t tt_launch_conv_fp32(const TTLaunch &L, cudaStream_t st);
// Uplink aggregation at a cell: output slot s = sum over members (in order) of their complex64
// output slot s, plus the cell's AWGN, then rounded and saturated (or stored as complex64).
struct TTCellMember {
  const float2 *ring_out;  // member's complex64 output ring [Q][n_rx][N]
  int ring_q;
  int pad;
};
struct TTCellArgs {
  void *ring_out;          // cell output ring [Q][n_rx][N] of packed int16 IQ (or complex64)
  const TTCellMember *members;
  int n_members, n, n_rx, ring_q, out_f32;
  uint32_t cell_id;
  uint64_t seed;
  float noise_std;         // sqrt(noise_var / 2), 0 = no AWGN
};
cudaError_t tt_launch_cell_reduce(const TTCellArgs &A, uint64_t first_slot, uint32_t n_slots, cudaStream_t st);
// Continuous CIR -> taps on the delay grid 0 .. n_taps-1: taps[t][link][k] = sum_p gains[t][link][p] *
// sinc(k - tau[t][p]), FP64 sums rounded to complex64.
// Sum-of-sinusoids anchors of one channel for slots [slot_first, slot_first + n_slots) (every
// symbol) plus, if tail, the first anchor of slot slot_first + n_slots, into its anchor ring.
struct TTSosJob {
  const TTUEDesc *ue;         // the channel's descriptor (device): N, symbols, symbol starts
  float2 *ring;               // [ring_len][per] anchors, anchor a at a % ring_len
  const float *amp;           // [per]
  const double *freq, *phase; // [per][m][2]
  double inv_fs;              // 1 / sample rate
  unsigned long long slot_first;
  unsigned long long thread_begin;  // first thread of this job in the launch
  int per, m, ring_len, n_slots, tail;
};
// One launch for every job: thread thread_begin + (slot - slot_first) * per + e of job j.
cudaError_t tt_launch_sos(const TTSosJob *jobs, int n_jobs, unsigned long long n_threads, cudaStream_t st);
// Timed traces (entries every `step` samples, e.g. 1 ms): before each run, the anchors of the slots
// it launches are interpolated in FP64 trace time from the stored trace into the channel's anchor
// ring, so the convolution kernels read per-symbol anchors.  One warp per (job, anchor): anchors
// 0 .. n_slots * nsym of the job, anchor k being a = slot_first * nsym + k; thread_begin counts warps.
struct TTRetimeJob {
  const TTUEDesc *ue;         // the channel's descriptor (device): N, symbols, symbol starts
  float2 *ring;               // [ring_len][per] anchors, anchor a at a % ring_len
  const float2 *src;          // [T][per] the stored trace
  double step;                // samples per stored entry
  unsigned long long T;       // stored entries
  unsigned long long slot_first;
  unsigned long long thread_begin;
  int loop, per, ring_len, n_slots;
};
cudaError_t tt_launch_retime(const TTRetimeJob *jobs, int n_jobs, unsigned long long n_warps, cudaStream_t st);
// Sparse convolution: for anchors [a_first, a_first + n_anchors) of one channel, the top_n taps of
// each link by binary32 power at the anchor (ties: lower index), compacted in tap order into the
// channel's sparse ring with (H, H[a+1] - H) and their delays; one warp per (anchor, link).
struct TTTopnJob {
  const TTUEDesc *ue;
  unsigned long long a_first;
  unsigned long long warp_begin;
  int n_anchors, links;
};
cudaError_t tt_launch_topn_select(const TTTopnJob *jobs, int n_jobs, unsigned long long n_warps, cudaStream_t st);
cudaError_t tt_launch_cir_resample(const float2 *gains, const double *tau, int n_steps, int n_links, int n_paths,
                                   int n_taps, float2 *taps, cudaStream_t st);

cudaError_t tt_launch_conv_s1(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s2(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s4(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s8(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s16(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s1_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s2_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s4_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s8_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s16_topn(const TTLaunch &L, cudaStream_t st);
// the same variants at TT_TPB_WIDE threads per CTA
cudaError_t tt_launch_conv_s1_w(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s2_w(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s4_w(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s8_w(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s16_w(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s1_w_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s2_w_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s4_w_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s8_w_topn(const TTLaunch &L, cudaStream_t st);
cudaError_t tt_launch_conv_s16_w_topn(const TTLaunch &L, cudaStream_t st);

// Block-Toeplitz tensor-core kernel (tcgen05, BF16 or FP16 operands): one work item per
// (UE, slot, symbol), in groups of up to 1536 samples; status is set to 1 if a bounded wait on the
// tensor core expires.  no_mma (tests only): the MMA warp issues no MMA, so the other roles' bounded
// waits run out with nothing in flight on the tensor core.
size_t tt_tc_smem_bytes();
int tt_tc_max_delay();
int tt_tc_items_per_slot(const int32_t *sym_len, int nsym);  // work items per slot of a channel
cudaError_t tt_launch_toeplitz_tc(const TTLaunch &L, bool fp16, int *status, int no_mma, cudaStream_t st);

// Record a message for tt_last_error() (thread-local) and return the status.
int32_t tt_set_error(int32_t status, const char *msg);

// Write the device's %globaltimer (ns) to dst once every earlier kernel on st has finished.
cudaError_t tt_launch_stamp(unsigned long long *dst, cudaStream_t st);

// Plain comparison form: one launch per UE per slot.
cudaError_t tt_launch_plain(const TTUEDesc *ue_dev, uint64_t slot, int n, cudaStream_t st);
