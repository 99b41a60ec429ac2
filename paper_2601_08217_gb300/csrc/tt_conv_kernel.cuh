// Tiled FP32 kernel for the per-UE time-varying channel convolution
//     y_r[m] = sum_t sum_k h_{r,t,k}(m) x_t[m - d_k] + w_r[m]        (Sec. III-B, y_u = x * h_u)
// with taps interpolated linearly between OFDM-symbol anchors taken from the
// UE's trace (Sec. IV), AWGN from Philox4x32-10, and int16 packing, all fused.
//
// Work decomposition.  A slot of one UE is cut into groups of S consecutive
// samples (S divides every symbol length, so a group never straddles a symbol
// and shares one set of taps).  A work item is TT_TPB consecutive groups of
// one (UE, slot): one CTA, one group per thread, all Rx antennas per thread so
// every staged input sample is reused n_rx times.
//
// Shared memory per item:
//   taps  float4 [symbols touched][NRX][n_tx][K] = (H[a], H[a+1] - H[a])  (interpolation endpoints)
//   offk  int    [K]  plane offset of each delay
//   planes float2 [n_tx][2S][NP]  the input window x[w_first - DP, w_last + S)
// The window is stored in 2S "phase planes": plane b holds the elements whose
// index is b mod S (planes S..2S-1 repeat planes 0..S-1 shifted by one row).
// Thread l needs x[S*l + j - d] for j = 0..S-1; in this layout those are
// plane (j - d mod S + S), row (l - floor(d/S) - ...), so for one delay all
// lanes read consecutive 8-byte words (conflict-free), and the S samples of a
// thread sit at a compile-time stride NP: one LDS with an immediate offset
// per tap-sample, no per-sample index arithmetic.
#pragma once

#include "tt_internal.h"
#include "tt_philox.cuh"

namespace tt {


// Anchor value H[a] for flat tap index e in [0, per) = ((r*n_tx + t)*K + k).
// step_samples == 0: trace entry a.  Otherwise: linear interpolation of the
// trace in FP64 time at the symbol's first sample (trace entry i at i*step).
__device__ __forceinline__ float2 tt_trace_entry(const TTUEDesc *__restrict__ U, uint64_t i, int e,
                                                 int per) {
  const uint64_t T = (uint64_t)U->n_anchors;
  const uint64_t idx = U->loop ? (i % T) : (i < T ? i : T - 1);
  return __ldg(U->taps + idx * (uint64_t)per + (uint64_t)e);
}

__device__ __forceinline__ float2 tt_anchor(const TTUEDesc *__restrict__ U, uint64_t a, int e, int per) {
  if (U->step_samples == 0.0) return tt_trace_entry(U, a, e, per);
  const uint64_t nsym = (uint64_t)U->nsym;
  const uint64_t b = (a / nsym) * (uint64_t)U->n + (uint64_t)U->sym_start[a % nsym];
  const double p = (double)b / U->step_samples;
  const double i0 = floor(p);
  const double f = p - i0;
  const float2 h0 = tt_trace_entry(U, (uint64_t)i0, e, per);
  const float2 h1 = tt_trace_entry(U, (uint64_t)i0 + 1, e, per);
  return make_float2((float)((double)h0.x + f * ((double)h1.x - (double)h0.x)),
                     (float)((double)h0.y + f * ((double)h1.y - (double)h0.y)));
}

// Stage the window x[ws, ws + wlen) of Tx antenna t into the phase planes.
// Element e goes to plane (e mod S) row (e / S) + 1 and plane (e mod S) + S row e / S.
template <int S, int NP>
__device__ __forceinline__ void tt_stage_window(float2 *__restrict__ pl, const uint32_t *__restrict__ rin,
                                                int ws, int wlen, int n, int n_tx, int t, int slot_pos, int Q,
                                                int tid) {
  if constexpr (S >= 4) {
    // four consecutive samples per thread: one 16-byte load, never straddling a slot
    for (int e = 4 * tid; e < wlen; e += 4 * TT_TPB) {
      int w = ws + e;
      int pos = slot_pos;
      if (w < 0) {  // delay line: earlier slots of this UE
        const int back = (-w + n - 1) / n;
        w += back * n;
        pos -= back;
        while (pos < 0) pos += Q;
      }
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(rin + ((size_t)(pos * n_tx + t) * n + w)));
      const int beta = e % S, i = e / S;
      const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 xv = tt_unpack_iq(vv[c]);
        pl[(beta + c) * NP + i + 1] = xv;
        pl[(beta + c + S) * NP + i] = xv;
      }
    }
  } else {
    for (int e = tid; e < wlen; e += TT_TPB) {
      int w = ws + e;
      int pos = slot_pos;
      if (w < 0) {
        const int back = (-w + n - 1) / n;
        w += back * n;
        pos -= back;
        while (pos < 0) pos += Q;
      }
      const float2 xv = tt_unpack_iq(__ldg(rin + ((size_t)(pos * n_tx + t) * n + w)));
      const int beta = e % S, i = e / S;
      pl[beta * NP + i + 1] = xv;
      pl[(beta + S) * NP + i] = xv;
    }
  }
}

template <int S, int NRX, int DMAX>
__global__ void __launch_bounds__(TT_TPB)
    tt_conv_fp32_kernel(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs, int n_segs,
                        uint32_t total_items, uint32_t *__restrict__ counter) {
  constexpr int NP = tt_geo_np(S, DMAX);
  constexpr int KU = S >= 16 ? 1 : 2;  // tap-loop unroll
  extern __shared__ float4 dyn_smem[];
  __shared__ uint32_t s_item;
  __shared__ int s_ue, s_g0, s_gend, s_jfirst, s_nsymt;
  __shared__ unsigned long long s_slot, s_idx0;
  __shared__ int s_sym[TT_MAX_SYM + 1];

  const int tid = threadIdx.x;
  uint32_t item = blockIdx.x;
  for (;;) {
    if (counter) {
      if (tid == 0) s_item = atomicAdd(counter, 1u);
      __syncthreads();
      item = s_item;
    }
    if (item >= total_items) return;

    // ---- locate the item: segment -> (UE, slot, first group); trace index of the first anchor ----
    if (tid == 0) {
      int lo = 0, hi = n_segs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
      }
      const TTSeg sg = segs[lo];
      const TTUEDesc *U = ues + sg.ue;
      const uint32_t rel = item - sg.item_begin;
      const uint32_t ips = (uint32_t)U->items_per_slot;
      const int g0 = (int)(rel % ips) * TT_TPB;
      const int gend = min(g0 + TT_TPB, U->groups);
      const int w0 = g0 * S, wl = (gend - 1) * S;
      int j = 0;
      while (j + 1 < U->nsym && U->sym_start[j + 1] <= w0) ++j;
      int jl = j;
      while (jl + 1 < U->nsym && U->sym_start[jl + 1] <= wl) ++jl;
      const uint64_t slot = sg.first_slot + rel / ips;
      const uint64_t a0 = slot * (uint64_t)U->nsym + (uint64_t)j;
      const uint64_t T = (uint64_t)U->n_anchors;
      s_idx0 = U->loop ? a0 % T : a0;
      s_slot = slot;
      s_ue = (int)sg.ue;
      s_g0 = g0;
      s_gend = gend;
      s_jfirst = j;
      s_nsymt = jl - j + 1;
    }
    __syncthreads();

    const TTUEDesc *__restrict__ U = ues + s_ue;
    const uint64_t slot = s_slot;
    const int g0 = s_g0, gend = s_gend, jf = s_jfirst, nst = s_nsymt;
    const int n = U->n, nsym = U->nsym, n_tx = U->n_tx, K = U->n_taps, Q = U->ring_q;
    const int dpad = U->dpad;
    const int per = NRX * n_tx * K;
    if (tid <= nsym) s_sym[tid] = U->sym_start[tid];

    float4 *tapsm = dyn_smem;
    const int ntap_e = nst * per;
    int *offk = reinterpret_cast<int *>(tapsm + ntap_e);
    float2 *planes = reinterpret_cast<float2 *>(offk + ((K + 3) & ~3));

    // ---- taps of the touched symbols: (H[a], H[a+1] - H[a]) ----
    if (U->step_samples == 0.0) {
      // one trace entry per symbol: entry index of anchor a0 + j without 64-bit division
      const uint64_t T = (uint64_t)U->n_anchors;
      const uint64_t idx0 = s_idx0;
      for (int e = tid; e < ntap_e; e += TT_TPB) {
        const int jl = e / per;
        const int rem = e - jl * per;
        uint64_t i0 = idx0 + (uint64_t)jl, i1 = i0 + 1;
        if (U->loop) {
          while (i0 >= T) i0 -= T;
          while (i1 >= T) i1 -= T;
        } else {
          i0 = i0 < T ? i0 : T - 1;
          i1 = i1 < T ? i1 : T - 1;
        }
        const float2 h0 = __ldg(U->taps + i0 * (uint64_t)per + (uint64_t)rem);
        const float2 h1 = __ldg(U->taps + i1 * (uint64_t)per + (uint64_t)rem);
        tapsm[e] = make_float4(h0.x, h0.y, h1.x - h0.x, h1.y - h0.y);
      }
    } else {
      for (int e = tid; e < ntap_e; e += TT_TPB) {
        const int jl = e / per;
        const int rem = e - jl * per;
        const uint64_t a = slot * (uint64_t)nsym + (uint64_t)(jf + jl);
        const float2 h0 = tt_anchor(U, a, rem, per);
        const float2 h1 = tt_anchor(U, a + 1, rem, per);
        tapsm[e] = make_float4(h0.x, h0.y, h1.x - h0.x, h1.y - h0.y);
      }
    }
    for (int k = tid; k < K; k += TT_TPB) {
      const int d = __ldg(U->delays + k);
      offk[k] = (S - d % S) * NP - d / S;
    }

    // ---- input window x[w_first - dpad, w_last + S) from the ring, int16 -> float ----
    const int ws = g0 * S - dpad;
    const int wlen = (gend - g0) * S + dpad;
    const int slot_pos = (int)(slot % (uint64_t)Q);
    const uint32_t *__restrict__ rin = reinterpret_cast<const uint32_t *>(U->ring_in);
    for (int t = 0; t < n_tx; ++t)
      tt_stage_window<S, NP>(planes + t * (2 * S * NP), rin, ws, wlen, n, n_tx, t, slot_pos, Q, tid);
    __syncthreads();

    // ---- S consecutive outputs per thread, all Rx antennas ----
    const int g = g0 + tid;
    if (g < gend) {
      const int w_me = g * S;
      int j = jf;
      while (j + 1 < nsym && s_sym[j + 1] <= w_me) ++j;
      const int o = w_me - s_sym[j];
      const float rL = 1.0f / (float)(s_sym[j + 1] - s_sym[j]);
      float tau[S];
#pragma unroll
      for (int jj = 0; jj < S; ++jj) tau[jj] = (float)(o + jj) * rL;

      float2 acc[NRX][S];
#pragma unroll
      for (int r = 0; r < NRX; ++r)
#pragma unroll
        for (int jj = 0; jj < S; ++jj) acc[r][jj] = make_float2(0.f, 0.f);

      const float4 *tb = tapsm + (j - jf) * per;
      const int q0 = tid + dpad / S;
      for (int t = 0; t < n_tx; ++t) {
        const float2 *pl = planes + t * (2 * S * NP) + q0;
        const float4 *tbt = tb + t * K;
#pragma unroll KU
        for (int k = 0; k < K; ++k) {
          const float2 *px = pl + offk[k];
          float2 xv[S];
#pragma unroll
          for (int jj = 0; jj < S; ++jj) xv[jj] = px[jj * NP];
#pragma unroll
          for (int r = 0; r < NRX; ++r) {
            const float4 h = tbt[r * n_tx * K + k];
#pragma unroll
            for (int jj = 0; jj < S; ++jj) {
              const float hr = fmaf(tau[jj], h.z, h.x);
              const float hi = fmaf(tau[jj], h.w, h.y);
              acc[r][jj].x = fmaf(hr, xv[jj].x, acc[r][jj].x);
              acc[r][jj].x = fmaf(-hi, xv[jj].y, acc[r][jj].x);
              acc[r][jj].y = fmaf(hr, xv[jj].y, acc[r][jj].y);
              acc[r][jj].y = fmaf(hi, xv[jj].x, acc[r][jj].y);
            }
          }
        }
      }

      // ---- epilogue: AWGN, pack, store ----
      const float nstd = U->noise_std;
      const uint64_t m0 = slot * (uint64_t)n + (uint64_t)w_me;
#pragma unroll
      for (int r = 0; r < NRX; ++r) {
        if (nstd > 0.f) {
          if (S == 1) {
            tt_awgn_add_one(U->seed, U->ue_id, (uint32_t)r, m0, nstd, acc[r][0]);
          } else {
#pragma unroll
            for (int jj = 0; jj < S; jj += 2)
              tt_awgn_add_pair(U->seed, U->ue_id, (uint32_t)r, m0 + (uint64_t)jj, nstd, acc[r][jj],
                               acc[r][jj + 1]);
          }
        }
        if (U->out_f32) {
          float2 *dstf = reinterpret_cast<float2 *>(U->ring_out) + ((size_t)(slot_pos * NRX + r) * n + w_me);
#pragma unroll
          for (int jj = 0; jj < S; ++jj) dstf[jj] = acc[r][jj];
          continue;
        }
        uint32_t pk[S];
#pragma unroll
        for (int jj = 0; jj < S; ++jj) pk[jj] = tt_pack_iq(acc[r][jj].x, acc[r][jj].y);
        uint32_t *dst = reinterpret_cast<uint32_t *>(U->ring_out) + ((size_t)(slot_pos * NRX + r) * n + w_me);
        if (S >= 4 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int jj = 0; jj < S; jj += 4)
            *reinterpret_cast<uint4 *>(dst + jj) = make_uint4(pk[jj], pk[jj + 1], pk[jj + 2], pk[jj + 3]);
        } else {
#pragma unroll
          for (int jj = 0; jj < S; ++jj) dst[jj] = pk[jj];
        }
      }
    }
    if (!counter) return;
    __syncthreads();
  }
}

template <int S, int NRX, int DMAX>
cudaError_t tt_launch_variant(const TTLaunch &L, cudaStream_t st) {
  auto kern = tt_conv_fp32_kernel<S, NRX, DMAX>;
  static bool attr_done = false;  // benign race: the attribute call is idempotent
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const unsigned grid = L.counter ? (unsigned)L.grid : L.total_items;
  if (grid == 0) return cudaSuccess;
  kern<<<grid, TT_TPB, L.smem, st>>>(L.ues, L.segs, L.n_segs, L.total_items, L.counter);
  return cudaGetLastError();
}

template <int S, int NRX, int DMAX>
int tt_occupancy_variant(size_t smem) {
  int blocks = 0;
  auto kern = tt_conv_fp32_kernel<S, NRX, DMAX>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, TT_TPB, smem) != cudaSuccess) return 1;
  return blocks > 0 ? blocks : 1;
}

template <int S, int NRX>
cudaError_t tt_launch_dclass(const TTLaunch &L, cudaStream_t st) {
  if (L.grid < 0) {  // occupancy query: blocks per SM returned through grid
    int b = 1;
    switch (L.dclass) {
      case 0: b = tt_occupancy_variant<S, NRX, TT_DCLASS0>(L.smem); break;
      case 1: b = tt_occupancy_variant<S, NRX, TT_DCLASS1>(L.smem); break;
      case 2: b = tt_occupancy_variant<S, NRX, TT_DCLASS2>(L.smem); break;
      default: return cudaErrorInvalidValue;
    }
    const_cast<TTLaunch &>(L).grid = -b;
    return cudaSuccess;
  }
  switch (L.dclass) {
    case 0: return tt_launch_variant<S, NRX, TT_DCLASS0>(L, st);
    case 1: return tt_launch_variant<S, NRX, TT_DCLASS1>(L, st);
    case 2: return tt_launch_variant<S, NRX, TT_DCLASS2>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int S>
cudaError_t tt_launch_spt(const TTLaunch &L, cudaStream_t st) {
  switch (L.nrx) {
    case 1: return tt_launch_dclass<S, 1>(L, st);
    case 2: return tt_launch_dclass<S, 2>(L, st);
    case 3:
      if constexpr (S <= 8) return tt_launch_dclass<S, 3>(L, st);
      return cudaErrorInvalidValue;
    case 4:
      if constexpr (S <= 8) return tt_launch_dclass<S, 4>(L, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tt
