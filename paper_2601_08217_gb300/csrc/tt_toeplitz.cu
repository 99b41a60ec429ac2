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
// Polyphase form (delay d = 8q + s, q = 0..15, s = 0..7, so d < 128):
//     D[m][n] = sum_{t, p, s, q'} X_{t,p,s}[m][q'] * W[n][(t,p,s,q')]
//     X_{t,p,s}[m][q'] = x_{t,p}[m - s - 120 + 8 q']          (q' = 15 - q; p = re/im part of x)
//     n = (r, output part, A or B): 16 rows for up to 4 Rx antennas
// For a fixed (t, p, s) the signal operand X is a Hankel-like view of one
// contiguous run of samples: element (m, q') sits at byte 2 m + 16 q' of a
// buffer holding x shifted by s.  That is exactly an MN-major shared-memory
// matrix descriptor with 8-element core matrices 16 bytes apart along M and
// 128 bytes apart along K, so the expanded Toeplitz operand is never stored:
// the tensor core reads the window itself.  Eight phase-shifted copies keep
// every descriptor start 16-byte aligned.  The tap operand W (16 x 1024) is
// built once per (UE, symbol) and reused by all of the symbol's 128-sample
// tiles.  One MMA per (t, p, s): M = 128 samples, N = 16, K = 16.
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

constexpr int kTPB = 128;
constexpr int kTile = 128;            // output samples per MMA tile (M)
constexpr int kPhases = 8;            // s
constexpr int kQ = 16;                // q' (delays < 8 * 16 = 128)
constexpr int kMaxDelayTC = kPhases * kQ - 1;
constexpr int kBufElems = 256;        // phase buffer: j = (m - m0) + 8 q' < 128 + 120
constexpr int kWin = kBufElems + 8;   // raw window samples per tile: phase buffer s reads raw[7 - s + j]
constexpr int kN = 16;                // D columns: (r, part, A|B)
constexpr int kKTot = 4 * 2 * kPhases * kQ;  // 1024: (t, p, s, q')
constexpr uint32_t kTmemCols = 32;
constexpr long long kSpinLimit = 1ll << 26;

// shared memory layout (bytes)
constexpr int kOffA = 0;                                          // [4 tx][2 parts][8 phases][256] x 2 B
constexpr int kOffW = kOffA + 4 * 2 * kPhases * kBufElems * 2;   // 32 KB: [2 n-groups][128 k-groups][8][8] x 2 B
constexpr int kOffTap = kOffW + kN * kKTot * 2;                  // [16 links][128 delays] float4
constexpr int kOffRaw = kOffTap + 16 * 128 * 16;                 // [4 tx][2 parts][kWin] float
constexpr int kSmemBytes = kOffRaw + 4 * 2 * kWin * 4;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading/stride byte offsets, no swizzle.
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

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool FP16>
__device__ __forceinline__ uint16_t to_op(float v) {
  if constexpr (FP16) return __half_as_ushort(__float2half_rn(v));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

struct TCItem {
  unsigned long long slot;
  int ue, sym, valid;
};

}  // namespace

template <bool FP16>
__global__ void __launch_bounds__(kTPB)
    tt_toeplitz_tc_kernel(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs, int n_segs,
                          uint32_t total_items, uint32_t *__restrict__ counter, int *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ TCItem s_it;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint16_t *Abuf = reinterpret_cast<uint16_t *>(sm + kOffA);
  uint16_t *Wbuf = reinterpret_cast<uint16_t *>(sm + kOffW);
  float4 *tapd = reinterpret_cast<float4 *>(sm + kOffTap);
  float *raw = reinterpret_cast<float *>(sm + kOffRaw);
  const uint32_t mbar = smem_u32(&s_mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    s_abort = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = s_tmem;
  uint32_t phase = 0;

  // idesc: D = F32, A/B = F16 (0) or BF16 (1), A MN-major, B K-major, N = 16, M = 128
  const uint32_t fmt = FP16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 15) | ((uint32_t)(kN >> 3) << 17) |
                         ((uint32_t)(kTile >> 4) << 24);

  uint32_t next_static = blockIdx.x;
  for (;;) {
    if (tid == 0) {
      const uint32_t item = counter ? atomicAdd(counter, 1u) : next_static;
      TCItem it{};
      it.valid = 0;
      if (item < total_items) {
        int lo = 0, hi = n_segs - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
        }
        const TTSeg sg = segs[lo];
        const uint32_t rel = item - sg.item_begin;
        const uint32_t nsym = (uint32_t)ues[sg.ue].nsym;
        it.slot = sg.first_slot + rel / nsym;
        it.sym = (int)(rel % nsym);
        it.ue = (int)sg.ue;
        it.valid = 1;
      }
      s_it = it;
    }
    next_static += gridDim.x;
    __syncthreads();
    const TCItem it = s_it;
    if (!it.valid || s_abort) break;
    const TTUEDesc *__restrict__ U = ues + it.ue;
    const int n = U->n, n_tx = U->n_tx, n_rx = U->n_rx, K = U->n_taps, Q = U->ring_q, nsym = U->nsym;
    const int sym0 = U->sym_start[it.sym], sym1 = U->sym_start[it.sym + 1];
    const int per = n_rx * n_tx * K;
    const int slot_pos = (int)(it.slot % (uint64_t)Q);
    const uint64_t a = it.slot * (uint64_t)nsym + (uint64_t)it.sym;

    // ---- dense delay table of this symbol: tapd[r*4+t][d] = (H, dH) ----
    for (int e = tid; e < 16 * 128; e += kTPB) tapd[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int e = tid; e < per; e += kTPB) {  // delays may repeat: accumulate
      const int k = e % K, rt = e / K, r = rt / n_tx, t = rt % n_tx;
      const int d = __ldg(U->delays + k);
      const float2 h0 = tt::tt_anchor(U, a, e, per);
      const float2 h1 = tt::tt_anchor(U, a + 1, e, per);
      float *v = reinterpret_cast<float *>(&tapd[(r * 4 + t) * 128 + d]);
      atomicAdd(v + 0, h0.x);
      atomicAdd(v + 1, h0.y);
      atomicAdd(v + 2, h1.x - h0.x);
      atomicAdd(v + 3, h1.y - h0.y);
    }
    __syncthreads();
    // ---- tap operand W[n][k], K-major, core matrices 8x8 (16 B rows): k-groups 128 B apart,
    //      n-groups 16 KB apart.  n = (r, out part, A|B), k = (t, p, s, q') ----
    for (int e = tid; e < kN * kKTot; e += kTPB) {
      const int nrow = e / kKTot, k = e % kKTot;
      const int r = nrow >> 2, op = (nrow >> 1) & 1, ab = nrow & 1;
      const int t = k >> 8, p = (k >> 7) & 1, s = (k >> 4) & 7, qp = k & 15;
      const int d = 8 * (15 - qp) + s;
      float v = 0.f;
      if (r < n_rx && t < n_tx) {
        const float4 h = tapd[(r * 4 + t) * 128 + d];
        const float hr = ab ? h.z : h.x, hi = ab ? h.w : h.y;
        // out re: re(x)*hr - im(x)*hi ; out im: re(x)*hi + im(x)*hr
        v = op == 0 ? (p == 0 ? hr : -hi) : (p == 0 ? hi : hr);
      }
      const int off = (nrow >> 3) * 16384 + (k >> 3) * 128 + (nrow & 7) * 16 + (k & 7) * 2;
      Wbuf[off >> 1] = to_op<FP16>(v);
    }

    // ---- 128-sample tiles of the symbol ----
    for (int m0 = sym0; m0 < sym1; m0 += kTile) {
      // raw window x_t[w], w in [m0 - 127, m0 - 127 + kWin), converted to float; zero beyond the slot
      const int wbase = m0 - 127;
      const uint32_t *__restrict__ rin = reinterpret_cast<const uint32_t *>(U->ring_in);
      for (int e = tid; e < n_tx * kWin; e += kTPB) {
        const int t = e / kWin, j = e % kWin;
        int w = wbase + j, pos = slot_pos;
        float2 xv = make_float2(0.f, 0.f);
        if (w < n) {
          if (w < 0) {
            const int back = (-w + n - 1) / n;
            w += back * n;
            pos -= back;
            while (pos < 0) pos += Q;
          }
          xv = tt_unpack_iq(__ldg(rin + ((size_t)(pos * n_tx + t) * n + w)));
        }
        raw[(t * 2 + 0) * kWin + j] = xv.x;
        raw[(t * 2 + 1) * kWin + j] = xv.y;
      }
      __syncthreads();
      // phase buffers: A_{t,p,s}[j] = x_{t,p}[m0 - s - 120 + j] = raw[(t,p)][7 - s + j]
      for (int e = tid; e < n_tx * 2 * kPhases * (kBufElems / 8); e += kTPB) {
        const int chunk = e % (kBufElems / 8), tps = e / (kBufElems / 8);
        const int s = tps % kPhases, tp = tps / kPhases;
        const float *src = raw + tp * kWin + (7 - s) + chunk * 8;
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          pk[i] = (uint32_t)to_op<FP16>(src[2 * i]) | ((uint32_t)to_op<FP16>(src[2 * i + 1]) << 16);
        *reinterpret_cast<uint4 *>(Abuf + tps * kBufElems + chunk * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        const uint32_t a_base = smem_u32(Abuf), w_base = smem_u32(Wbuf);
        const int nmma = n_tx * 2 * kPhases;
        for (int i = 0; i < nmma; ++i) {
          const uint64_t ad = umma_desc(a_base + (uint32_t)i * kBufElems * 2, /*lbo K*/ 128, /*sbo M*/ 16);
          const uint64_t bd = umma_desc(w_base + (uint32_t)i * 2 * 128, /*lbo K*/ 128, /*sbo N*/ 16384);
          umma_f16(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
        }
        umma_commit(mbar);
      }
      // wait for the tile's MMAs (bounded); lane 0 of each warp polls, the warp follows its verdict
      int done = 0;
      if (lane == 0) {
        long long spins = 0;
        while (!(done = mbar_try_wait(mbar, phase)) && ++spins < kSpinLimit) {
        }
        if (!done) {
          atomicExch(status, 1);
          s_abort = 1;
        }
      }
      done = __shfl_sync(0xFFFFFFFFu, done, 0);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      if (done) {
        // epilogue: lane = sample m0 + 32 warp + lane; 16 accumulator columns
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
        const int m = m0 + warp * 32 + lane;
        if (m < sym1) {
          const float tau = (float)(m - sym0) / (float)(sym1 - sym0);
          const uint64_t mabs = it.slot * (uint64_t)n + (uint64_t)m;
          for (int r = 0; r < n_rx; ++r) {
            float2 y = make_float2(fmaf(tau, v[r * 4 + 1], v[r * 4 + 0]), fmaf(tau, v[r * 4 + 3], v[r * 4 + 2]));
            if (U->noise_std > 0.f) tt_awgn_add_one(U->seed, U->ue_id, (uint32_t)r, mabs, U->noise_std, y);
            const size_t o = (size_t)(slot_pos * n_rx + r) * n + m;
            if (U->out_f32) reinterpret_cast<float2 *>(U->ring_out)[o] = y;
            else reinterpret_cast<uint32_t *>(U->ring_out)[o] = tt_pack_iq(y.x, y.y);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      __syncthreads();
      if (s_abort) break;
    }
    if (s_abort) break;
  }
  __syncthreads();
  if (s_abort && tid == 0) {  // one more bounded wait for anything still in flight
    long long spins = 0;
    while (!mbar_try_wait(mbar, phase) && ++spins < kSpinLimit) {
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

size_t tt_tc_smem_bytes() { return (size_t)kSmemBytes; }
int tt_tc_max_delay() { return kMaxDelayTC; }

cudaError_t tt_launch_toeplitz_tc(const TTLaunch &L, bool fp16, int *status, cudaStream_t st) {
  auto kern = fp16 ? tt_toeplitz_tc_kernel<true> : tt_toeplitz_tc_kernel<false>;
  static bool attr[2] = {false, false};
  if (!attr[fp16]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    attr[fp16] = true;
  }
  if (L.grid < 0) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kTPB, kSmemBytes) != cudaSuccess) blocks = 1;
    const_cast<TTLaunch &>(L).grid = -(blocks > 0 ? blocks : 1);
    return cudaSuccess;
  }
  if (L.grid == 0 || L.total_items == 0) return cudaSuccess;
  kern<<<L.grid, kTPB, kSmemBytes, st>>>(L.ues, L.segs, L.n_segs, L.total_items, L.counter, status);
  return cudaGetLastError();
}
