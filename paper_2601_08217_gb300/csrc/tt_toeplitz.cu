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
//     D[c][(i, n)] = sum_{t, p, j} X_{t,p}[c][j] * W[(i, n)][(t, p, j)]
//     X_{t,p}[c][j] = x_{t,p}[8 c + j - 128],     W[(i, n)][(t, p, j)] = tap of delay i + 128 - j
//     c = block row (M), i = sample in the block, n = (r, output part, A or B), p = re/im part of x
// so output sample 8 c + i of (r, part) is D[c][(i, n)].  X is a Hankel-like
// view of one contiguous run of 16-bit samples: element (c, j) sits at byte
// 16 c + 2 j.  That is a K-major shared-memory matrix descriptor whose 8-row
// core matrices are 128 bytes apart along M and only 16 bytes apart along K,
// so the Toeplitz-expanded operand is never stored: the tensor core reads the
// staged window itself.  The tap operand W (128 x 1152 for 4 Tx) is too big to
// keep, so it streams in 4 KB K-chunks built in shared memory while the tensor
// core consumes the previous chunk; each chunk feeds up to four 128x128x16 MMAs
// (1024 samples each) whose accumulators fill the 512 tensor-memory columns.
//
// Every wait on the MMA-completion barrier is bounded; on expiry the kernel
// sets the status word to 1, frees its tensor memory and exits.
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
constexpr int kRows = 128;            // block rows per MMA tile (M): 1024 samples
constexpr int kTilesMax = 2;          // tiles accumulating at once: 2 x 128 TMEM columns
constexpr int kGroup = kRows * kB * kTilesMax;  // samples per group (2048)
constexpr int kMaxDelayTC = 127;
constexpr int kW = 144;               // window per (t, p): j in [0, 135) used, padded to 9 K-chunks of 16
constexpr int kKC = kW / 16;          // K-chunks per (t, p)
constexpr int kN = 128;               // D columns: (i, r, part, A|B)
constexpr int kSig = kGroup + kW;     // staged samples per (t, p)
constexpr uint32_t kTmemCols = kTilesMax * kN;  // two CTAs per SM share the 512 columns
constexpr long long kSpinLimit = 1ll << 24;

constexpr int kQW = 88;               // words per component table: q = j - i + 8 in [1, 151] needs 76, plus shift <= 3
constexpr int kComps = 4;             // hr, hi of H and of dH; -hi is hi with the sign bits flipped
constexpr int kPer = 4;               // tap chunks per pipeline step
constexpr int kSteps = 2;             // steps in the ring: builders run up to one step ahead of the MMAs
constexpr int kStages = kPer * kSteps;
constexpr int kChunkBytes = kN * 16 * 2;

// shared memory layout (bytes).  The dense delay table is only read while the component tables
// are built, before any signal is staged for the item, so it shares the signal's space.
constexpr int kOffSig = 0;                               // [4 tx][2 parts][kSig] 16-bit operands
constexpr int kOffTap = 0;                               // [16 links][128 delays] float4 (H, dH), by tap_pos(d)
constexpr int kOffW = kOffSig + 4 * 2 * kSig * 2;        // kStages x 4 KB tap chunks: [16 n-groups][2 k-groups][8][8]
constexpr int kOffComp = kOffW + kStages * kChunkBytes;  // [4 tx][2 parities][kComps][4 rx][kQW words]
constexpr int kSmemUsed = kOffComp + 16 * kComps * 2 * kQW * 4;
static_assert(16 * 128 * 16 <= 4 * 2 * kSig * 2, "delay table must fit in the signal area");

// Component tables, one per (t, parity, c, r), kQW words each.  A builder warp handles one sample i
// of the block and all 16 rows (r, output part, A|B) for both K-groups (4 words apart); for either
// input part it reads, at one (t, parity), the four tables c of every r.  Table (t, par, c, r) starts
// at word ((t * 2 + par) * 4 + c) * 4 + r) * kQW, whose bank is 24 r (mod 32) because kQW = 88 is
// 24 mod 32; shifting its data by c words puts the warp's 32 words of every 32-bit load on 32
// distinct banks.
__host__ __device__ constexpr int comp_slot(int t, int par, int c, int r) { return ((t * 2 + par) * kComps + c) * 4 + r; }
static_assert(kQW % 32 == 24 && 76 + (kComps - 1) <= kQW, "component table stride and shift");
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

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
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
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase)
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

template <bool FP16>
__global__ void __launch_bounds__(kTPB, 2)
    tt_toeplitz_tc_kernel(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs, int n_segs,
                          uint32_t total_items, uint32_t *__restrict__ counter, int *__restrict__ status) {
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
  uint16_t *wbuf = reinterpret_cast<uint16_t *>(sm + kOffW);
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
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&s_full[b])), "n"(kBuildWarps));
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

  // idesc: D = F32, A/B = F16 (0) or BF16 (1), both K-major, N = 128, M = 128
  const uint32_t fmt = FP16 ? 0u : 1u;
  const uint32_t idesc =
      (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  const uint32_t sig_base = smem_u32(sig), w_base = smem_u32(wbuf);

  // this builder thread's fixed segment of every tap chunk: row (i, r, part, A|B), k-group kg.
  // Lanes 8h .. 8h + 7 of a warp take rows 8 (h >> 1) .. + 7 of its 16 and k-group h & 1, so each
  // quarter-warp stores one contiguous 128-byte run of the chunk.
  const int row = warp * 16 + ((lane >> 4) << 3) + (lane & 7), kg = (lane >> 3) & 1;
  const int ii = row >> 4, nn = row & 15, rr = nn >> 2, op = (nn >> 1) & 1, ab = nn & 1;
  const int qoff = kg * 8 - ii + 8, par = qoff & 1;
  // (op, p) -> component: (0,0) hr, (0,1) -hi, (1,0) hi, (1,1) hr
  const int c_p0 = ab * 2 + (op == 0 ? 0 : 1), c_p1 = ab * 2 + (op == 0 ? 1 : 0);
  const uint32_t neg_p1 = op == 0 ? 0x80008000u : 0u;
  const int w_off = ((row >> 3) * 256 + kg * 128 + (row & 7) * 16) / 2;

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
      const uint64_t bdesc0 = umma_desc(w_base, /*lbo K*/ 128, /*sbo N*/ 256);
      const uint64_t adesc0 = umma_desc(sig_base, /*lbo K*/ 16, /*sbo M*/ 128);
      for (int gs = sym0; gs < sym1; gs += kGroup) {
        const int blocks = (min(gs + kGroup, sym1) - gs + kB - 1) / kB;
        const int n_tiles = (blocks + kRows - 1) / kRows;
        if (ggroup > 0) warp_wait(smem_u32(&s_tfree), (ggroup - 1) & 1u, status, abort_flag);
        int tp = 0, jc = jlo;
        for (int s = 0; s < steps; ++s, ++gstep) {
          const uint32_t ss = gstep % kSteps;
          warp_wait(smem_u32(&s_full[ss]), (gstep / kSteps) & 1u, status, abort_flag);
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          if (lane == 0) {
            const int kk0 = s * kPer, kend = min(kk0 + kPer, nk);
            uint64_t bd = bdesc0 + (uint64_t)((ss * kPer * kChunkBytes) >> 4);
            for (int kk = kk0; kk < kend; ++kk) {
              // signal view: element (row c, k) at 16 c + 2 k from the tile's first sample, k from 16 jc
              const uint64_t ad = adesc0 + (uint64_t)(((tp * kSig + jc * 16) * 2) >> 4);
              const uint32_t acc = kk > 0 ? 1u : 0u;
              // tiles are 2048 bytes of signal apart
              if (n_tiles > 1) umma_f16(tmem + kN, ad + 128, bd, idesc, acc);
              umma_f16(tmem, ad, bd, idesc, acc);
              bd += kChunkBytes >> 4;
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
        uint32_t *dst = comp_w + slot * kQW + c;
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
      // table word bases of this thread's segment for input part p (Tx antenna added per chunk)
      // (rows of absent Rx antennas read table r = 0 and write zeros)
      const int rq = rr < n_rx ? rr : 0;
      const uint32_t keep = rr < n_rx ? 0xFFFFFFFFu : 0u;
      const int tb0 = comp_slot(0, par, c_p0, rq) * kQW + c_p0 + (qoff - par) / 2;
      const int tb1 = comp_slot(0, par, c_p1, rq) * kQW + c_p1 + (qoff - par) / 2;

      // ---- the symbol in groups of up to 4096 samples (4 tensor-memory tiles each) ----
      for (int gs = sym0; gs < sym1; gs += kGroup) {
        const int ge = min(gs + kGroup, sym1);
        const int blocks = (ge - gs + kB - 1) / kB;
        const int n_tiles = (blocks + kRows - 1) / kRows;
        // signal: sig[t][p][u] = x_{t,p}[gs - 128 + u], 16-bit operands, zero past the slot end;
        // four samples per load (the window start is 8-aligned and N is a multiple of 8).  The
        // accumulators of the previous group are complete, so nothing reads the old signal.
        {
          const uint32_t *__restrict__ rin = reinterpret_cast<const uint32_t *>(U->ring_in);
          const int quads = (n_tiles * kRows * kB + kW) / 4;
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
        // tap chunks, kPer per step, into the step's ring slots once the MMAs of the step that
        // last used them are done; each warp then arrives on the step's full barrier
        int tp = 0, jc = jlo;
        for (int s = 0; s < steps; ++s, ++gstep) {
          const uint32_t ss = gstep % kSteps;
          if (gstep >= kSteps) warp_wait(smem_u32(&s_empty[ss]), (gstep / kSteps - 1) & 1u, status, abort_flag);
          const int kk0 = s * kPer, kend = min(kk0 + kPer, nk);
          uint16_t *wdst = wbuf + ss * kPer * (kN * 16) + w_off;
#pragma unroll
          for (int e = 0; e < kPer; ++e) {
            if (kk0 + e < kend) {
              const int t = tp >> 1, p = tp & 1;
              const uint32_t *src = comp_w + (p ? tb1 : tb0) + t * (2 * kComps * 4 * kQW) + jc * 8;
              const uint32_t ng = p ? neg_p1 : 0u;
              *reinterpret_cast<uint4 *>(wdst + e * (kN * 16)) =
                  make_uint4((src[0] ^ ng) & keep, (src[1] ^ ng) & keep, (src[2] ^ ng) & keep, (src[3] ^ ng) & keep);
              if (++jc == kKC) { jc = jlo; ++tp; }
            }
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&s_full[ss]));
        }
        // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (block rows) and samples
        //      i in [4 (w / 4), 4 (w / 4) + 4) of each block; AWGN per pair of samples (one Philox block) ----
        warp_wait(smem_u32(&s_acc), ggroup & 1u, status, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        {
          const int quad = warp & 3, ihalf = warp >> 2;
          const float rl = 1.0f / (float)(sym1 - sym0);
          for (int mt = 0; mt < n_tiles; ++mt) {
            const int c = mt * kRows + quad * 32 + lane;
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(mt * kN + ihalf * 4 * 16);
#pragma unroll
            for (int q = 0; q < 4; q += 2) {
              uint32_t v0[16], v1[16];  // samples i and i + 1 of this lane's block row: 16 columns each
              tmem_ld16(tbase + (uint32_t)q * 16, v0);
              tmem_ld16(tbase + (uint32_t)(q + 1) * 16, v1);
              tmem_wait_ld();
              const int i = ihalf * 4 + q;
              const int m = gs + c * kB + i;  // even: pairs (m, m + 1) share a Philox block
              if (m < ge) {
                const float tau0 = (float)(m - sym0) * rl, tau1 = (float)(m + 1 - sym0) * rl;
                const uint64_t mabs = it.slot * (uint64_t)n + (uint64_t)m;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  if (r >= n_rx) break;
                  float2 y0 = make_float2(fmaf(tau0, __uint_as_float(v0[r * 4 + 1]), __uint_as_float(v0[r * 4 + 0])),
                                          fmaf(tau0, __uint_as_float(v0[r * 4 + 3]), __uint_as_float(v0[r * 4 + 2])));
                  float2 y1 = make_float2(fmaf(tau1, __uint_as_float(v1[r * 4 + 1]), __uint_as_float(v1[r * 4 + 0])),
                                          fmaf(tau1, __uint_as_float(v1[r * 4 + 3]), __uint_as_float(v1[r * 4 + 2])));
                  if (U->noise_std > 0.f)
                    tt_awgn_add_pair(U->seed, U->ue_id, (uint32_t)r, mabs, U->noise_std, y0, y1);
                  const size_t o = (size_t)(slot_pos * n_rx + r) * n + m;
                  if (U->out_f32) {
                    *reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(U->ring_out) + o) =
                        make_float4(y0.x, y0.y, y1.x, y1.y);
                  } else {
                    *reinterpret_cast<uint2 *>(reinterpret_cast<uint32_t *>(U->ring_out) + o) =
                        make_uint2(tt_pack_iq(y0.x, y0.y), tt_pack_iq(y1.x, y1.y));
                  }
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
  return nsym;  // one work item per symbol; its samples run in groups of up to 4096
}

cudaError_t tt_launch_toeplitz_tc(const TTLaunch &L, bool fp16, int *status, cudaStream_t st) {
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
  kern<<<L.grid, kTPB, kSmemBytes, st>>>(L.ues, L.segs, L.n_segs, L.total_items, L.counter, status);
  return cudaGetLastError();
}
