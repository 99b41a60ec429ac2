// Block-Toeplitz tensor-core form of the per-UE channel convolution
// (Sec. III-B, y_u = x * h_u), for dense multi-antenna channels, on the 5th
// generation tensor cores (tcgen05.mma, kind::f16: BF16 or FP16 operands,
// FP32 accumulation in tensor memory).
//
// Inside one OFDM symbol the interpolated taps split exactly:
//     y_r[m] = A_r[m] + tau(m) B_r[m],
//     A_r[m] = sum_t sum_d H_{r,t}(d) x_t[m-d],   B_r[m] = sum_t sum_d dH_{r,t}(d) x_t[m-d],
// with H = the symbol's anchor and dH = next anchor - anchor: two static
// convolutions whose sum over delays is a matrix product.
//
// Block form (blocks of 8 output samples, delays d < 128):
//     D[(i, n)][c] = sum_{t, p, j} W[(i, n)][(t, p, j)] * X_{t,p}[c][j]
//     X_{t,p}[c][j] = x_{t,p}[8 c + j - 128],     W[(i, n)][(t, p, j)] = tap of delay i + 128 - j
//     c = block row, i = sample in the block, n = (r, output part, A or B), p = re/im part of x
// so output sample 8 c + i of (r, part) is D[(i, n)][c].  X is a Hankel-like
// view of one contiguous run of 16-bit samples: element (c, j) sits at byte
// 16 c + 2 j.  That is a K-major shared-memory matrix descriptor whose 8-row
// core matrices are 128 bytes apart along N and only 16 bytes apart along K,
// so the Toeplitz-expanded signal is never stored: the tensor core reads the
// staged window itself (the B operand, N = up to 192 block rows, 1536 samples).
//
// The tap operand W (128 rows x 1152 for 4 Tx) is the A operand and lives in
// tensor memory: builder warps expand each 16-wide K-chunk from compact
// component tables straight into a ring of tensor-memory columns
// (tcgen05.st), so the only shared-memory traffic of an MMA is its signal
// view and the builders' table reads.  Accumulators take 192 of the CTA's
// 256 tensor-memory columns, the chunk ring the other 64; two CTAs share an
// SM.
//
// Every wait on an mbarrier is bounded; on expiry the kernel sets the status
// word to 1, frees its tensor memory and exits.
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tt_conv_kernel.cuh"
#include "tt_internal.h"
#include "tt_philox.cuh"

namespace {

constexpr int kBuildWarps = 8;                  // stage, build tap chunks, epilogue
constexpr int kTPB = (kBuildWarps + 1) * 32;    // + one warp that issues the MMAs
constexpr int kBuilders = kBuildWarps * 32;
constexpr int kB = 8;                 // output samples per block row (16-byte rows of the signal view)
constexpr int kM = 128;               // D rows: (i, r, part, A|B)
constexpr int kNMax = 192;            // D columns per group: block rows (1536 samples)
constexpr int kGroup = kNMax * kB;    // samples per group
constexpr int kMaxDelayTC = 127;
constexpr int kW = 144;               // window per (t, p): j in [0, 135) used, padded to 9 K-chunks of 16
constexpr int kKC = kW / 16;          // K-chunks per (t, p)
constexpr int kSig = kGroup + kW;     // staged samples per (t, p)
constexpr uint32_t kTmemCols = 256;   // two CTAs per SM share the 512 columns
constexpr uint32_t kAccCols = kNMax;  // accumulator columns [0, 192)
constexpr uint32_t kChunkCols = 8;    // one K-chunk of A: 128 lanes x 16 16-bit values
// Bounded waits: each poll may suspend the thread for up to kSuspendNs until the phase completes
// (the thread wakes when it does), so 2^20 polls bound a wait at about one second.
constexpr long long kSpinLimit = 1ll << 20;
constexpr uint32_t kSuspendNs = 1000;

constexpr int kQW = 88;               // words per component table: q = j - i + 8 in [1, 151] needs 76, plus shift <= 8
constexpr int kComps = 4;             // hr, hi of H and of dH; -hi is hi with the sign bits flipped
constexpr int kPer = 4;               // tap chunks per pipeline step
constexpr int kSteps = 2;             // steps in the ring: builders run up to one step ahead of the MMAs
constexpr int kStages = kPer * kSteps;
static_assert(kAccCols + kStages * kChunkCols <= kTmemCols, "accumulators and chunk ring fit the allocation");

// shared memory layout (bytes).  The dense delay table is only read while the component tables
// are built, before any signal is staged for the item, so it shares the signal's space.
constexpr int kOffSig = 0;                               // [4 tx][2 parts][kSig] 16-bit operands
constexpr int kOffTap = 0;                               // [16 links][128 delays] float4 (H, dH), by tap_pos(d)
constexpr int kSigBytes = 4 * 2 * kSig * 2;
constexpr int kTapBytes = 16 * 128 * 16;
constexpr int kOffComp = kSigBytes > kTapBytes ? kSigBytes : kTapBytes;  // [4 tx][2 parities][kComps][4 rx][kQW words]
constexpr int kSmemUsed = kOffComp + 16 * kComps * 2 * kQW * 4;

// Component tables, one per (t, parity, c, r), kQW words each.  Table (t, par, c, r) starts at
// word ((t * 2 + par) * 4 + c) * 4 + r) * kQW, whose bank is 24 r (mod 32) because kQW = 88 is
// 24 mod 32, and its data is shifted by c + 5 par words.  A builder warp's 32 rows are two samples
// i (of opposite parity, whose word offsets differ by one), four Rx antennas and four components:
// their words land on banks 24 r + c + 4 par + const, all 32 distinct.
__host__ __device__ constexpr int comp_slot(int t, int par, int c, int r) { return ((t * 2 + par) * kComps + c) * 4 + r; }
__host__ __device__ constexpr int comp_shift(int c, int par) { return c + 5 * par; }
static_assert(kQW % 32 == 24 && 76 + comp_shift(kComps - 1, 1) <= kQW, "component table stride and shift");
// Two CTAs per SM (each with half the tensor-memory columns): one stages, builds tables or drains
// its accumulators while the other keeps the tensor core busy.  A third never fits.
constexpr int kSmemBytes = kSmemUsed;
constexpr int kCtasPerSm = 2;
static_assert(kCtasPerSm * (int)kTmemCols <= 512, "tensor-memory columns of the co-resident CTAs");
static_assert(3 * (kSmemBytes + 2048) > 228 * 1024 && 2 * (kSmemBytes + 2048) <= 228 * 1024,
              "exactly two CTAs per SM");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Position of delay d in a link's row of the dense delay table: even delays first, then odd ones,
// so the table build, which reads delays two apart across a warp, reads consecutive entries.
__device__ __forceinline__ int tap_pos(int d) { return (d >> 1) | ((d & 1) << 6); }

// Shared-memory matrix descriptor: start, leading/stride byte offsets, no swizzle.  The start
// address sits in the low 14 bits (16-byte units), so adding (bytes >> 4) moves the start.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;
}

// D (tensor memory) (+)= A (tensor memory, M = 128 lanes x K = 16) * B (shared-memory descriptor)^T
__device__ __forceinline__ void umma_f16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// builder-warp barrier (named barrier 1): the MMA warp is not stopped
__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kBuilders) : "memory"); }

// 16 consecutive accumulator columns of this thread's lane; completes at tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// The same wait, tied to the 16 registers of an earlier tmem_ld16 so that no use of them is
// scheduled before the data has arrived.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// 4 consecutive columns of this thread's lane (32-bit each); complete at tmem_wait_st().  It touches
// tensor memory only (no memory clobber), so the shared-memory loads of later chunks may be issued
// ahead of it; tcgen05.wait::st orders it before the step's barrier arrival.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(taddr), "r"(a), "r"(b), "r"(c),
               "r"(d));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Transpose of a 4 x 4 block held by lanes 4g .. 4g + 3 (lane 4g + j holds row j in v): afterwards
// lane 4g + j holds column j, v[s] = row s's element j.  Two butterfly exchanges.
__device__ __forceinline__ void transpose4(float v[4], int j) {
  const bool b1 = (j & 2) != 0, b0 = (j & 1) != 0;
  float x0 = b1 ? v[0] : v[2], x1 = b1 ? v[1] : v[3];
  float y0 = __shfl_xor_sync(0xFFFFFFFFu, x0, 2), y1 = __shfl_xor_sync(0xFFFFFFFFu, x1, 2);
  float a0 = b1 ? y0 : v[0], a1 = b1 ? y1 : v[1], a2 = b1 ? v[2] : y0, a3 = b1 ? v[3] : y1;
  x0 = b0 ? a0 : a1;
  x1 = b0 ? a2 : a3;
  y0 = __shfl_xor_sync(0xFFFFFFFFu, x0, 1);
  y1 = __shfl_xor_sync(0xFFFFFFFFu, x1, 1);
  v[0] = b0 ? y0 : a0;
  v[1] = b0 ? a1 : y0;
  v[2] = b0 ? y1 : a2;
  v[3] = b0 ? a3 : y1;
}

template <bool FP16>
__device__ __forceinline__ uint16_t to_op(float v) {
  if constexpr (FP16) return __half_as_ushort(__float2half_rn(v));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

struct TCItem {
  unsigned long long slot;
  unsigned long long idx0, idx1;  // trace entries of the symbol's anchor and the next one
  int ue, sym, valid;
};

// Bounded wait on an mbarrier phase by the whole warp: lane 0 polls, the warp follows its verdict.
// Once any wait of the CTA has expired (abort flag), every later wait returns at once, so each
// role runs through its remaining steps without blocking and the CTA reaches its exit.
__device__ __forceinline__ void warp_wait(uint32_t mbar, uint32_t phase, int *status, volatile int *abort_flag) {
  if ((threadIdx.x & 31) == 0) {
    long long spins = 0;
    bool done = false;
    while (!(done = mbar_try_wait(mbar, phase)) && !*abort_flag && ++spins < kSpinLimit) {
    }
    if (!done && !*abort_flag) {
      atomicExch(status, 1);
      *abort_flag = 1;
    }
  }
  __syncwarp();
}

}  // namespace

// Two CTAs per SM: 18 warps, five on some SM sub-partition, whose 16,384 registers then allow 96 a
// thread (5 warps x 32 x 96 = 15,360); the launch bounds give the compiler that limit.
template <bool FP16>
__global__ void __launch_bounds__(kTPB, 2)
    tt_toeplitz_tc_kernel(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs, int n_segs,
                          uint32_t total_items, uint32_t *__restrict__ counter, int *__restrict__ status,
                          int no_mma, TTCheck ck) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) unsigned long long s_full[kSteps];   // builders -> MMA warp: step's chunks written
  __shared__ __align__(8) unsigned long long s_empty[kSteps];  // MMA completion -> builders: step's slots free
  __shared__ __align__(8) unsigned long long s_acc;            // MMA completion of a group -> epilogue
  __shared__ __align__(8) unsigned long long s_tfree;          // epilogue done with the accumulators -> MMA warp
  __shared__ __align__(8) unsigned long long s_drain;          // the MMA thread's last commit -> tensor memory free
  __shared__ uint32_t s_tmem;
  __shared__ TCItem s_it;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint16_t *sig = reinterpret_cast<uint16_t *>(sm + kOffSig);
  float4 *tapd = reinterpret_cast<float4 *>(sm + kOffTap);
  uint32_t *comp_w = reinterpret_cast<uint32_t *>(sm + kOffComp);
  volatile int *abort_flag = &s_abort;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    for (int b = 0; b < kSteps; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&s_full[b])), "n"(kBuildWarps / 2));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_acc)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&s_tfree)), "n"(kBuildWarps));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s_drain)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = s_tmem;

  // idesc: D = F32, A/B = F16 (0) or BF16 (1), both K-major, M = 128; N (bits 17..22) per group
  const uint32_t fmt = FP16 ? 0u : 1u;
  const uint32_t idesc0 = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kM >> 4) << 24);
  const uint32_t sig_base = smem_u32(sig);

  // this builder thread's row of every tap chunk in tensor memory: lane 32 (warp % 4) + lane, row
  // (i, r, part, A|B) = that lane; warps w and w + 4 write K-halves kg = w / 4 of the same lanes
  const int quad = warp & 3, kg = warp >> 2;
  const int row = quad * 32 + lane;
  const int ii = row >> 4, nn = row & 15, rr = nn >> 2, op = (nn >> 1) & 1, ab = nn & 1;
  const int qoff = 8 - ii, par = qoff & 1;  // K-half 0; half 1 is the next 4 words of the tables
  // (op, p) -> component: (0,0) hr, (0,1) -hi, (1,0) hi, (1,1) hr
  const int c_p0 = ab * 2 + (op == 0 ? 0 : 1), c_p1 = ab * 2 + (op == 0 ? 1 : 0);
  const uint32_t neg_p1 = op == 0 ? 0x80008000u : 0u;
  const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);  // this warp's lanes, column 0

  uint32_t gstep = 0;  // pipeline steps since launch (both roles count them alike)
  uint32_t ggroup = 0; // accumulator groups since launch
  uint32_t next_static = blockIdx.x;
  for (;;) {
    if (tid == 0) {
      const uint32_t item = *abort_flag ? total_items : (counter ? atomicAdd(counter, 1u) : next_static);
      TCItem it{};
      it.valid = 0;
      if (item < total_items) {
        int lo = 0, hi = n_segs - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
        }
        const TTSeg sg = segs[lo];
        const TTUEDesc *U = ues + sg.ue;
        const uint32_t rel = item - sg.item_begin;
        const uint32_t nsym = (uint32_t)U->nsym;
        it.slot = sg.first_slot + rel / nsym;
        it.ue = (int)sg.ue;
        it.sym = (int)(rel % nsym);
        const uint64_t a0 = it.slot * (uint64_t)nsym + (uint64_t)it.sym, T = (uint64_t)U->n_anchors;
        it.idx0 = U->loop ? a0 % T : (a0 < T ? a0 : T - 1);
        it.idx1 = U->loop ? (a0 + 1) % T : (a0 + 1 < T ? a0 + 1 : T - 1);
        it.valid = 1;
      }
      s_it = it;
    }
    next_static += gridDim.x;
    __syncthreads();
    const TCItem it = s_it;
    if (!it.valid) break;
    const TTUEDesc *__restrict__ U = ues + it.ue;
    const int n = U->n, n_tx = U->n_tx, n_rx = U->n_rx, Q = U->ring_q;
    const int sym0 = U->sym_start[it.sym], sym1 = U->sym_start[it.sym + 1];
    const int slot_pos = (int)(it.slot % (uint64_t)Q);
    // K-chunks jc < jlo of every (t, p) window hold no tap: j = i + 128 - d >= 128 - d_max
    const int jlo = (128 - U->d_max) >> 4, kpc = kKC - jlo;
    const int nk = n_tx * 2 * kpc;  // K-chunks per group
    const int steps = (nk + kPer - 1) / kPer;

    if (warp == kBuildWarps) {
      // ================= MMA warp: lane 0 issues, the warp waits =================
      for (int gs = sym0; gs < sym1; gs += kGroup) {
        const int blocks = (min(gs + kGroup, sym1) - gs + kB - 1) / kB;
        const int ncols = (blocks + 15) & ~15;  // N: a multiple of 16 for M = 128
        const uint32_t idesc = idesc0 | ((uint32_t)(ncols >> 3) << 17);
        if (ggroup > 0) warp_wait(smem_u32(&s_tfree), (ggroup - 1) & 1u, status, abort_flag);
        // signal view: element (block row c, k) at 16 c + 2 k bytes from the window of (t, p) at 16 jc
        const uint64_t bdesc0 = umma_desc(sig_base, /*lbo K*/ 16, /*sbo N*/ 128);
        int tp = 0, jc = jlo;
        for (int s = 0; s < steps; ++s, ++gstep) {
          const uint32_t ss = gstep % kSteps;
          warp_wait(smem_u32(&s_full[ss]), (gstep / kSteps) & 1u, status, abort_flag);
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          if (lane == 0 && !no_mma) {
            const int kk0 = s * kPer, kend = min(kk0 + kPer, nk);
            uint32_t ta = tmem + kAccCols + ss * (kPer * kChunkCols);
            for (int kk = kk0; kk < kend; ++kk) {
              const uint64_t bd = bdesc0 + (uint64_t)(((tp * kSig + jc * 16) * 2) >> 4);
              umma_f16_ta(tmem, ta, bd, idesc, kk > 0 ? 1u : 0u);
              ta += kChunkCols;
              if (++jc == kKC) { jc = jlo; ++tp; }
            }
            umma_commit(smem_u32(&s_empty[ss]));
            if (s == steps - 1) umma_commit(smem_u32(&s_acc));
          }
          __syncwarp();
        }
        ++ggroup;
      }
    } else {
      // ================= builder warps =================
      const int per = n_rx * n_tx * U->n_taps, K = U->n_taps;
      const uint64_t a = it.slot * (uint64_t)U->nsym + (uint64_t)it.sym;
      // ---- dense delay table of this symbol: tapd[r*4+t][d] = (H, dH) ----
      for (int e = tid; e < 16 * 128; e += kBuilders) tapd[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      builders_sync();
      for (int rt = warp; rt < n_rx * n_tx; rt += kBuildWarps) {
        const int r = rt / n_tx, t = rt - r * n_tx;
#pragma unroll 4
        for (int k = lane; k < K; k += 32) {  // delays may repeat: accumulate
          const int e = rt * K + k;
          const int d = __ldg(U->delays + k);
          if (!TT_IN(d >= 0 && d <= kMaxDelayTC, TT_CHK_TAP_SMEM)) continue;
          if (!TT_IN(U->step_samples != 0.0 ||
                         (it.idx0 < (uint64_t)U->n_anchors && it.idx1 < (uint64_t)U->n_anchors),
                     TT_CHK_TAP_GLOBAL))
            continue;
          float2 h0, h1;
          if (U->step_samples == 0.0) {
            h0 = __ldg(U->taps + it.idx0 * (uint64_t)per + (uint64_t)e);
            h1 = __ldg(U->taps + it.idx1 * (uint64_t)per + (uint64_t)e);
          } else {
            h0 = tt::tt_anchor(U, a, e, per);
            h1 = tt::tt_anchor(U, a + 1, e, per);
          }
          float *v = reinterpret_cast<float *>(&tapd[(r * 4 + t) * 128 + tap_pos(d)]);
          atomicAdd(v + 0, h0.x);
          atomicAdd(v + 1, h0.y);
          atomicAdd(v + 2, h1.x - h0.x);
          atomicAdd(v + 3, h1.y - h0.y);
        }
      }
      builders_sync();
      // ---- component tables: 16-bit c-component of the tap of delay 136 - (q + par), per
      //      (t, par, c, r) slot of kQW words at shift c; two q per 32-bit store ----
      for (int slot = warp; slot < 16 * kComps * 2; slot += kBuildWarps) {
        const int r = slot & 3, c = (slot >> 2) & (kComps - 1), tpar = (slot >> 4) & 1, t = slot >> 5;
        uint32_t *dst = comp_w + slot * kQW + comp_shift(c, tpar);
        const float4 *tl = tapd + (r * 4 + t) * 128;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int qh = lane + 32 * j;
          if (qh < 76) {
            uint32_t pk = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int d = 136 - (2 * qh + h + tpar);
              float v = 0.f;
              if (d >= 0 && d <= 127) {
                const float4 tv = tl[tap_pos(d)];
                const float2 hv = (c & 2) ? make_float2(tv.z, tv.w) : make_float2(tv.x, tv.y);
                v = (c & 1) ? hv.y : hv.x;
              }
              pk |= (uint32_t)to_op<FP16>(v) << (16 * h);
            }
            dst[qh] = pk;
          }
        }
      }
      builders_sync();
      // table word bases of this thread's row for input part p (Tx antenna added per chunk)
      // (rows of absent Rx antennas read table r = 0 and write zeros)
      const int rq = rr < n_rx ? rr : 0;
      const uint32_t keep = rr < n_rx ? 0xFFFFFFFFu : 0u;
      const int tb0 = comp_slot(0, par, c_p0, rq) * kQW + comp_shift(c_p0, par) + (qoff - par) / 2;
      const int tb1 = comp_slot(0, par, c_p1, rq) * kQW + comp_shift(c_p1, par) + (qoff - par) / 2;

      // ---- the symbol in groups of up to kGroup samples (one accumulator of up to 192 columns) ----
      for (int gs = sym0; gs < sym1; gs += kGroup) {
        const int ge = min(gs + kGroup, sym1);
        const int blocks = (ge - gs + kB - 1) / kB;
        const int ncols = (blocks + 15) & ~15;
        // signal: sig[t][p][u] = x_{t,p}[gs - 128 + u], 16-bit operands, zero past the slot end;
        // four samples per load (the window start is 8-aligned and N is a multiple of 8).  The
        // accumulators of the previous group are complete, so nothing reads the old signal.
        {
          const uint32_t *__restrict__ rin = reinterpret_cast<const uint32_t *>(U->ring_in);
          const int quads = (ncols * kB + kW) / 4;
#pragma unroll 2
          for (int qd = tid; qd < quads; qd += kBuilders) {
            const int u = qd * 4;
            int w = gs - 128 + u, pos = slot_pos;
            const bool live = w < n;
            if (live && w < 0) {
              const int back = (-w + n - 1) / n;
              w += back * n;
              pos -= back;
              while (pos < 0) pos += Q;
            }
            const uint4 *src = reinterpret_cast<const uint4 *>(rin + ((size_t)pos * n_tx * n + w));
            if (!TT_IN(!live || (pos >= 0 && pos < Q && w >= 0 && w + 4 <= n), TT_CHK_RING_IN)) continue;
            if (!TT_IN(u + 4 <= kSig, TT_CHK_RAW_WRITE)) continue;
            uint4 v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t)
              v[t] = (live && t < n_tx) ? __ldg(src + (size_t)t * (n / 4)) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              if (t >= n_tx) break;
              const uint32_t vv[4] = {v[t].x, v[t].y, v[t].z, v[t].w};
              uint32_t re2[2], im2[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float2 x0 = tt_unpack_iq(vv[2 * h]), x1 = tt_unpack_iq(vv[2 * h + 1]);
                re2[h] = (uint32_t)to_op<FP16>(x0.x) | ((uint32_t)to_op<FP16>(x1.x) << 16);
                im2[h] = (uint32_t)to_op<FP16>(x0.y) | ((uint32_t)to_op<FP16>(x1.y) << 16);
              }
              *reinterpret_cast<uint2 *>(sig + (t * 2 + 0) * kSig + u) = make_uint2(re2[0], re2[1]);
              *reinterpret_cast<uint2 *>(sig + (t * 2 + 1) * kSig + u) = make_uint2(im2[0], im2[1]);
            }
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the signal, for the tensor core
        builders_sync();  // a step's arrivals come from one group: every warp's staging must be done
        // tap chunks, kPer per step, into the step's ring columns once the MMAs of the step that
        // last used them are done; each warp then arrives on the step's full barrier
        // Builder group kg (warps 4 kg .. 4 kg + 3) fills the steps with gstep % 2 == kg, both K-halves
        // of its lanes' rows, so two steps' load, store and wait chains run at once.
        int tp = 0, jc = jlo;
        for (int s = 0; s < steps; ++s, ++gstep) {
          const uint32_t ss = gstep % kSteps;
          const int kk0 = s * kPer, kend = min(kk0 + kPer, nk);
          const uint32_t *srcs[kPer];
          uint32_t ngs[kPer];
#pragma unroll
          for (int e = 0; e < kPer; ++e) {
            const int t = tp >> 1, p = tp & 1;
            srcs[e] = comp_w + (p ? tb1 : tb0) + t * (2 * kComps * 4 * kQW) + jc * 8;
            ngs[e] = p ? neg_p1 : 0u;
            if (kk0 + e + 1 < kend && ++jc == kKC) { jc = jlo; ++tp; }
          }
          if (kend - kk0 == kPer && ++jc == kKC) { jc = jlo; ++tp; }  // advance past the step's last chunk
          if ((int)(gstep & 1u) != kg) continue;                   // the other group's step
          if (gstep >= kSteps) {
            warp_wait(smem_u32(&s_empty[ss]), (gstep / kSteps - 1) & 1u, status, abort_flag);
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          }
          const uint32_t tdst = t_row + kAccCols + ss * (kPer * kChunkCols);
#pragma unroll
          for (int e = 0; e < kPer; ++e) {
            const long long off = srcs[e] - comp_w;
            if (!TT_IN(off >= 0 && off + 8 <= 16 * kComps * 2 * kQW, TT_CHK_TAP_READ)) srcs[e] = comp_w;
          }
#pragma unroll
          for (int e = 0; e < kPer; ++e) {
            if (kk0 + e >= kend) break;
            uint32_t wv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) wv[q] = (srcs[e][q] ^ ngs[e]) & keep;
            if (TT_IN(kAccCols + ss * (kPer * kChunkCols) + e * kChunkCols + 8 <= kTmemCols, TT_CHK_TMEM))
              tmem_st8(tdst + e * kChunkCols, wv);
          }
          tmem_wait_st();
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s_full[ss]));
        }
        // ---- epilogue: warp w reads its lanes (rows 32 (w % 4) ..: samples i = 2 (w % 4) + lane / 16,
        //      Rx r = (lane / 4) % 4, (part, A|B) = lane % 4) over every other 16-column chunk, starting
        //      at chunk w / 4.  A 4 x 4 transpose among lanes 4g .. 4g + 3 gives lane 4g + j the four
        //      (part, A|B) values of block row c0 + j; lanes l and l ^ 16 hold samples i and i + 1,
        //      which share a Philox block.  Each lane computes one block per two block rows. ----
        warp_wait(smem_u32(&s_acc), ggroup & 1u, status, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        {
          const int j4 = lane & 3, hi16 = lane >> 4, r = (lane >> 2) & 3;
          const int i_me = quad * 2 + hi16;
          const float rl = 1.0f / (float)(sym1 - sym0);
          const bool live_r = r < n_rx;
          const float nstd = U->noise_std;
          for (int cc = kg; cc * 16 < ncols; cc += 2) {
            uint32_t raw[16];
            tmem_ld16(t_row + (uint32_t)(cc * 16), raw);
            tmem_wait_ld16(raw);
            // block quads (0, 1) and (2, 3): lane l computes the Philox block of its (r, sample pair)
            // at quad 2h + hi16 and trades half of it with lane l ^ 16
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float u[2][4];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
#pragma unroll
                for (int q = 0; q < 4; ++q) u[e][q] = __uint_as_float(raw[(2 * h + e) * 4 + q]);
                transpose4(u[e], j4);
              }
              const int c_mine = cc * 16 + (2 * h + hi16) * 4 + j4;      // block row of the block I compute
              const int m_pair = gs + c_mine * kB + quad * 2;              // even sample of that pair
              uint4 wv = make_uint4(0u, 0u, 0u, 0u);
              if (nstd > 0.f && live_r) {
                const uint64_t pabs = (it.slot * (uint64_t)n + (uint64_t)m_pair) >> 1;
                wv = tt_philox4x32_10(make_uint4((uint32_t)pabs, (uint32_t)(pabs >> 32), U->ue_id, (uint32_t)r),
                                      (uint32_t)U->seed, (uint32_t)(U->seed >> 32));
              }
              // hi16 = 0 keeps words 0, 1 (its even sample) of its own block, quad 2h; hi16 = 1 keeps
              // words 2, 3 (its odd sample) of its own block, quad 2h + 1
              const uint32_t s0 = hi16 ? wv.x : wv.z, s1 = hi16 ? wv.y : wv.w;
              const uint32_t g0 = __shfl_xor_sync(0xFFFFFFFFu, s0, 16), g1 = __shfl_xor_sync(0xFFFFFFFFu, s1, 16);
              // my sample at quad 2h (uses the partner's block when hi16 = 1) and at quad 2h + 1
              float2 y[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int qd = 2 * h + e;
                const int c = cc * 16 + qd * 4 + j4;
                const int m = gs + c * kB + i_me;
                const float tau = (float)(m - sym0) * rl;
                y[e] = make_float2(fmaf(tau, u[e][1], u[e][0]), fmaf(tau, u[e][3], u[e][2]));
                if (nstd > 0.f) {
                  // words of my sample: quad 2h + hi16 is my own block, the other quad the partner's
                  const bool own = e == hi16;
                  const uint32_t w0 = own ? (hi16 ? wv.z : wv.x) : g0, w1 = own ? (hi16 ? wv.w : wv.y) : g1;
                  tt_box_muller_add(w0, w1, nstd, y[e]);
                }
              }
              // lane l (hi16 = 0) stores the pair (i, i + 1) of quad 2h, lane l ^ 16 that of quad 2h + 1
              const float2 give = hi16 ? y[0] : y[1];
              const float2 got = make_float2(__shfl_xor_sync(0xFFFFFFFFu, give.x, 16),
                                             __shfl_xor_sync(0xFFFFFFFFu, give.y, 16));
              const float2 ylo = hi16 ? got : y[0], yhi = hi16 ? y[1] : got;  // samples i_even, i_even + 1
              const int c_st = cc * 16 + (2 * h + hi16) * 4 + j4;
              const int m_st = gs + c_st * kB + quad * 2;
              if (live_r && c_st < blocks && m_st < ge &&
                  TT_IN(m_st >= 0 && m_st + 2 <= n &&
                            (int64_t)(slot_pos * n_rx + r) * n + m_st + 2 <= (int64_t)Q * n_rx * n - ck.shrink,
                        TT_CHK_RING_OUT)) {
                const size_t o = (size_t)(slot_pos * n_rx + r) * n + m_st;
                if (U->out_f32) {
                  *reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(U->ring_out) + o) =
                      make_float4(ylo.x, ylo.y, yhi.x, yhi.y);
                } else {
                  *reinterpret_cast<uint2 *>(reinterpret_cast<uint32_t *>(U->ring_out) + o) =
                      make_uint2(tt_pack_iq(ylo.x, ylo.y), tt_pack_iq(yhi.x, yhi.y));
                }
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_tfree));
        ++ggroup;
      }
    }
  }
  // Before tensor memory is freed, the MMA thread commits once more: that commit arrives when every MMA
  // it issued has completed.  Normally the epilogues have waited for all of them already; after an
  // expired wait some may still run, so this wait is bounded but does not stop at the abort flag.
  if (warp == kBuildWarps && lane == 0) {
    umma_commit(smem_u32(&s_drain));
    long long spins = 0;
    while (!mbar_try_wait(smem_u32(&s_drain), 0) && ++spins < kSpinLimit) {
    }
    if (spins >= kSpinLimit) atomicExch(status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

size_t tt_tc_smem_bytes() { return (size_t)kSmemBytes; }
int tt_tc_max_delay() { return kMaxDelayTC; }
int tt_tc_items_per_slot(const int32_t *sym_len, int nsym) {
  (void)sym_len;
  return nsym;  // one work item per symbol; its samples run in groups of up to 1536
}

cudaError_t tt_launch_toeplitz_tc(const TTLaunch &L, bool fp16, int *status, int no_mma, cudaStream_t st) {
  auto kern = fp16 ? tt_toeplitz_tc_kernel<true> : tt_toeplitz_tc_kernel<false>;
  static bool attr[2] = {false, false};
  if (!attr[fp16]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr[fp16] = true;
  }
  if (L.grid < 0) {
    // The occupancy calculator reports one CTA per SM for any kernel that allocates tensor memory.
    // Shared memory admits exactly two of these CTAs per SM (static_assert above) and each takes
    // half of the 512 columns, so two run side by side.
    const_cast<TTLaunch &>(L).grid = -kCtasPerSm;
    return cudaSuccess;
  }
  if (L.grid == 0 || L.total_items == 0) return cudaSuccess;
  kern<<<L.grid, kTPB, kSmemBytes, st>>>(L.ues, L.segs, L.n_segs, L.total_items, L.counter, status, no_mma,
                                         L.check);
  return cudaGetLastError();
}
