// Tiled FP32 kernel for the per-UE time-varying channel convolution
//     y_r[m] = sum_t sum_k h_{r,t,k}(m) x_t[m - d_k] + w_r[m]        (Sec. III-B, y_u = x * h_u)
// with taps interpolated linearly between OFDM-symbol anchors taken from the
// UE's trace (Sec. IV), AWGN from Philox4x32-10, and int16 packing, all fused.
//
// Work decomposition.  A slot of one UE is cut into groups of S consecutive
// samples (S divides every symbol length, so a group never straddles a symbol
// and shares one set of taps).  A work item is TPB consecutive groups of
// one (UE, slot), TPB being the CTA's thread count (128 or 256): one group per
// thread, all Rx antennas per thread so every staged input sample is reused
// n_rx times.  The item's span TPB * S samples is the kernel's tile.
//
// Persistent, software-pipelined CTAs.  While a CTA computes item i it has
// already issued cp.async copies of item i+1's raw input window, raw trace
// entries and delays into shared memory, so global-memory latency overlaps
// the arithmetic; after a barrier the raw window is converted to float and
// scattered into the phase planes.
//
// Shared memory:
//   planes float2 [n_tx][2S][NP]  the input window x[w_first - dpad, w_last + S)
//   raw    uint32 [n_tx][WMAX]    the same window as packed int16 I/Q (cp.async target)
//   taps   float4 [2][tap_max]    (H[a], H[a+1] - H[a]) per touched symbol, double-buffered
//   dly    int    [2][k_max]      raw delays (cp.async target), then plane offsets
// The window is stored in 2S "phase planes": plane b holds the elements whose
// index is b mod S (planes S..2S-1 repeat planes 0..S-1 shifted by one row).
// Thread l needs x[S*l + j - d] for j = 0..S-1; in this layout those sit in
// plane (j - d mod S + S), row l - floor(d/S) + const, so for one delay all
// lanes read consecutive 8-byte words (conflict-free), and the S samples of a
// thread sit at a compile-time stride NP: one LDS with an immediate offset
// per tap-sample and no per-sample index arithmetic.
#pragma once

#include "tt_internal.h"
#include "tt_philox.cuh"

namespace tt {

// Index tests of the bounds-checked build: TT_IN(cond, code) is cond there (a false cond is
// recorded), and true without evaluating cond in the normal build.
#if defined(TT_CHECKED) && TT_CHECKED
__device__ __forceinline__ bool tt_chk(bool ok, const TTCheck &ck, uint32_t code) {
  if (!ok && ck.report && atomicAdd(ck.report, 1u) == 0u) atomicExch(ck.report + 1, code);
  return ok;
}
#define TT_IN(cond, code) tt::tt_chk((cond), ck, (code))
#else
#define TT_IN(cond, code) true
#endif

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

// ---- small PTX helpers ----
__device__ __forceinline__ uint32_t tt_smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tt_cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(tt_smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void tt_cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(tt_smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void tt_cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(tt_smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void tt_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void tt_cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Packed pair FMA (two independent single-rounding FMAs, one instruction): a*b + c.
__device__ __forceinline__ float2 tt_fma2(float2 a, float2 b, float2 c) {
  uint64_t ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}

// Per-item description shared through smem.
struct TTItem {
  unsigned long long slot;
  unsigned long long idx0;  // trace entry of the item's first anchor (per-symbol traces)
  int ue, g0, gend, jf, nst, valid;
  int slot_pos;             // ring position of the slot: slot mod ring_q (once per item, not per thread)
};


// Thread 0: item index -> (UE, slot, groups, first symbol, symbols touched).
// With device cursors (graph replay), a run's first slot is cursors[ue] instead of seg.first_slot.
template <int TPB>
__device__ __forceinline__ void tt_locate(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs,
                                          int n_segs, uint32_t item, uint32_t total_items,
                                          const unsigned long long *__restrict__ cursors, TTItem &it) {
  if (item >= total_items) {
    it.valid = 0;
    return;
  }
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
  }
  const TTSeg sg = segs[lo];
  const TTUEDesc *U = ues + sg.ue;
  const uint32_t rel = item - sg.item_begin;
  const uint32_t ips = (uint32_t)U->items_per_slot;
  const uint32_t c = rel % ips;
  const int ci = __ldg(U->chunk_info + c);
  const int g0 = (int)c * TPB;
  const uint64_t slot = (cursors ? cursors[sg.ue] : sg.first_slot) + rel / ips;
  const int jf = ci & 0xFFFF;
  const uint64_t a0 = slot * (uint64_t)U->nsym + (uint64_t)jf;
  it.slot = slot;
  it.idx0 = U->loop ? a0 % (uint64_t)U->n_anchors : a0;
  it.ue = (int)sg.ue;
  it.g0 = g0;
  it.gend = min(g0 + TPB, U->groups);
  it.jf = jf;
  it.nst = ci >> 16;
  it.slot_pos = (int)(slot % (uint64_t)U->ring_q);
  it.valid = 1;
}

// All threads: start the asynchronous copies of one item's raw window, trace
// entries, delays and symbol table into shared memory.
template <int S, int NRX, bool TOPN, int TPB>
__device__ __forceinline__ void tt_issue_item(const TTUEDesc *__restrict__ U, const TTItem &it, uint32_t *raw,
                                              int wmax, float4 *taps, int *dly, int *sym, int tid,
                                              const TTCheck &ck) {
  const int n = U->n, n_tx = U->n_tx, Q = U->ring_q, K = U->n_taps, dpad = U->dpad;
  const int ws = it.g0 * S - dpad;
  const int wlen = (it.gend - it.g0) * S + dpad;
  const int slot_pos = it.slot_pos;
  const uint32_t *__restrict__ rin = reinterpret_cast<const uint32_t *>(U->ring_in);
  constexpr int V = S >= 4 ? 4 : 1;  // samples per copy: 16-byte copies when windows are 4-aligned
  for (int t = 0; t < n_tx; ++t) {
    uint32_t *rt = raw + t * wmax;
    for (int e = V * tid; e < wlen; e += V * TPB) {
      int w = ws + e;
      int pos = slot_pos;
      if (w < 0) {  // delay line: earlier slots of this UE
        const int back = (-w + n - 1) / n;
        w += back * n;
        pos -= back;
        while (pos < 0) pos += Q;
      }
      const uint32_t *src = rin + ((size_t)(pos * n_tx + t) * n + w);
      if (!TT_IN(e + V <= wmax, TT_CHK_RAW_WRITE)) continue;
      if (!TT_IN(pos >= 0 && pos < Q && w >= 0 && w + V <= n, TT_CHK_RING_IN)) continue;
      if (V == 4) tt_cp_async16(rt + e, src); else tt_cp_async4(rt + e, src);
    }
  }
  const int per = NRX * n_tx * K;
  const int ntap_e = it.nst * per;
  if constexpr (TOPN) {
    // sparse convolution: the kept taps of each touched symbol and link, selected ahead of the run
    const int ns = NRX * n_tx * U->top_n;
    const uint64_t L = (uint64_t)U->sparse_len;
    for (int e = tid; e < it.nst * ns; e += TPB) {
      const int jl = e / ns;
      const int rem = e - jl * ns;
      const uint64_t a = it.slot * (uint64_t)U->nsym + (uint64_t)(it.jf + jl);
      const size_t src = (size_t)(a % L) * ns + rem;
      if (!TT_IN(e < ck.tap_max, TT_CHK_TAP_SMEM) || !TT_IN(e < ck.kpad, TT_CHK_DLY_SMEM)) continue;
      if (!TT_IN(src < L * (uint64_t)ns, TT_CHK_TAP_GLOBAL)) continue;
      tt_cp_async16(&taps[e], U->sparse + src);
      tt_cp_async4(dly + e, U->sparse_dly + src);
    }
    if (tid <= U->nsym && TT_IN(tid <= TT_MAX_SYM, TT_CHK_SYM)) tt_cp_async4(sym + tid, U->sym_start + tid);
    tt_cp_async_commit();
    return;
  }
  if (U->step_samples == 0.0) {
    const uint64_t T = (uint64_t)U->n_anchors;
    for (int e = tid; e < ntap_e; e += TPB) {
      const int jl = e / per;
      const int rem = e - jl * per;
      uint64_t i0 = it.idx0 + (uint64_t)jl, i1 = i0 + 1;
      if (U->loop) {
        while (i0 >= T) i0 -= T;
        while (i1 >= T) i1 -= T;
      } else {
        i0 = i0 < T ? i0 : T - 1;
        i1 = i1 < T ? i1 : T - 1;
      }
      if (!TT_IN(e < ck.tap_max, TT_CHK_TAP_SMEM) || !TT_IN(i0 < T && i1 < T, TT_CHK_TAP_GLOBAL)) continue;
      tt_cp_async8(&taps[e].x, U->taps + i0 * (uint64_t)per + (uint64_t)rem);
      tt_cp_async8(&taps[e].z, U->taps + i1 * (uint64_t)per + (uint64_t)rem);
    }
  }
  for (int k = tid; k < K; k += TPB)
    if (TT_IN(k < ck.kpad, TT_CHK_DLY_SMEM)) tt_cp_async4(dly + k, U->delays + k);
  if (tid <= U->nsym && TT_IN(tid <= TT_MAX_SYM, TT_CHK_SYM)) tt_cp_async4(sym + tid, U->sym_start + tid);
  tt_cp_async_commit();
}

// All threads, after the copies landed: raw window -> phase planes, taps -> (H0, dH),
// delays -> plane offsets.
template <int S, int NRX, int NP, bool TOPN, int WMAXC, int TPB>
__device__ __forceinline__ void tt_convert_item(const TTUEDesc *__restrict__ U, const TTItem &it,
                                                const uint32_t *raw, int wmax, float2 *planes, float4 *taps,
                                                int *dly, int tid, const TTCheck &ck) {
  const int n_tx = U->n_tx, K = U->n_taps, dpad = U->dpad;
  const int wlen = (it.gend - it.g0) * S + dpad;
  for (int t = 0; t < n_tx; ++t) {
    const uint32_t *rt = raw + t * wmax;
    float2 *pl = planes + t * (2 * S * NP);
    if constexpr (S >= 16) {
      // every 16-byte load of the thread first (at most NV), then the unpacking and plane stores (at
      // S = 8 under the 64-register bound of the single-antenna variants this spills: loop form below)
      constexpr int NV = (WMAXC + 4 * TPB - 1) / (4 * TPB);
      uint4 v[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int e = 4 * tid + q * 4 * TPB;
        if (e < wlen && TT_IN(e + 4 <= wmax, TT_CHK_RAW_READ)) v[q] = *reinterpret_cast<const uint4 *>(rt + e);
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int e = 4 * tid + q * 4 * TPB;
        if (e < wlen) {
          const uint32_t vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
          const int beta = e % S, i = e / S;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float2 xv = tt_unpack_iq(vv[c]);
            if (!TT_IN(beta + c < S && i + 1 < NP, TT_CHK_PLANE_WRITE)) continue;
            pl[(beta + c) * NP + i + 1] = xv;
            pl[(beta + c + S) * NP + i] = xv;
          }
        }
      }
    } else if constexpr (S >= 4) {
      for (int e = 4 * tid; e < wlen; e += 4 * TPB) {
        if (!TT_IN(e + 4 <= wmax, TT_CHK_RAW_READ)) continue;
        const uint4 v = *reinterpret_cast<const uint4 *>(rt + e);
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
        const int beta = e % S, i = e / S;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 xv = tt_unpack_iq(vv[c]);
          if (!TT_IN(beta + c < S && i + 1 < NP, TT_CHK_PLANE_WRITE)) continue;
          pl[(beta + c) * NP + i + 1] = xv;
          pl[(beta + c + S) * NP + i] = xv;
        }
      }
    } else {
      for (int e = tid; e < wlen; e += TPB) {
        if (!TT_IN(e < wmax, TT_CHK_RAW_READ)) continue;
        const float2 xv = tt_unpack_iq(rt[e]);
        const int beta = e % S, i = e / S;
        if (!TT_IN(i + 1 < NP, TT_CHK_PLANE_WRITE)) continue;
        pl[beta * NP + i + 1] = xv;
        pl[(beta + S) * NP + i] = xv;
      }
    }
  }
  if constexpr (TOPN) {  // (H, dH) came from the selection; delays become plane offsets
    for (int e = tid; e < it.nst * NRX * n_tx * U->top_n; e += TPB) {
      if (!TT_IN(e < ck.kpad, TT_CHK_DLY_SMEM)) continue;
      const int d = dly[e];
      dly[e] = (S - d % S) * NP - d / S;
    }
    return;
  }
  const int per = NRX * n_tx * K;
  const int ntap_e = it.nst * per;
  if (U->step_samples == 0.0) {
    for (int e = tid; e < ntap_e; e += TPB) {
      if (!TT_IN(e < ck.tap_max, TT_CHK_TAP_SMEM)) continue;
      float4 h = taps[e];
      h.z -= h.x;
      h.w -= h.y;
      taps[e] = h;
    }
  } else {  // trace-time interpolation (FP64) straight from global memory
    const int nsym = U->nsym;
    for (int e = tid; e < ntap_e; e += TPB) {
      const int jl = e / per;
      const int rem = e - jl * per;
      const uint64_t a = it.slot * (uint64_t)nsym + (uint64_t)(it.jf + jl);
      const float2 h0 = tt_anchor(U, a, rem, per);
      const float2 h1 = tt_anchor(U, a + 1, rem, per);
      if (!TT_IN(e < ck.tap_max, TT_CHK_TAP_SMEM)) continue;
      taps[e] = make_float4(h0.x, h0.y, h1.x - h0.x, h1.y - h0.y);
    }
  }
  for (int k = tid; k < K; k += TPB) {
    if (!TT_IN(k < ck.kpad, TT_CHK_DLY_SMEM)) continue;
    const int d = dly[k];
    dly[k] = (S - d % S) * NP - d / S;
  }
}

// All threads: S consecutive outputs per thread of one item, all Rx antennas, fused epilogue.
template <int S, int NRX, int NP, bool TOPN>
__device__ __forceinline__ void tt_compute_item(const TTUEDesc *__restrict__ U, const TTItem &it,
                                                const float2 *planes, const float4 *taps, const int *offk,
                                                const int *sym, int tid, const TTCheck &ck) {
  constexpr int KU = S >= 16 ? 1 : 2;  // tap-loop unroll
  const int g = it.g0 + tid;
  if (g >= it.gend) return;
  const int n = U->n, nsym = U->nsym, n_tx = U->n_tx, K = U->n_taps;
  const int per = NRX * n_tx * K;
  const int w_me = g * S;
  int j = it.jf;
  while (j + 1 < nsym && sym[j + 1] <= w_me) ++j;
  if (!TT_IN(j + 1 <= TT_MAX_SYM && j >= it.jf && j < it.jf + it.nst, TT_CHK_SYM)) return;
  const int o = w_me - sym[j];
  const float rL = 1.0f / (float)(sym[j + 1] - sym[j]);
  float2 tau2[S];  // (tau, tau) per sample: operand of the packed interpolation
#pragma unroll
  for (int jj = 0; jj < S; ++jj) {
    const float tv = (float)(o + jj) * rL;
    tau2[jj] = make_float2(tv, tv);
  }
  float2 acc[NRX][S];
#pragma unroll
  for (int r = 0; r < NRX; ++r)
#pragma unroll
    for (int jj = 0; jj < S; ++jj) acc[r][jj] = make_float2(0.f, 0.f);

  const int q0 = tid + U->dpad / S;
  if constexpr (TOPN) {
    // sparse convolution: the compacted top-n list of this symbol, per link, with its own offsets
    const int nsel = U->top_n;
    const float4 *tb = taps + (j - it.jf) * NRX * n_tx * nsel;
    const int *ob = offk + (j - it.jf) * NRX * n_tx * nsel;
    for (int t = 0; t < n_tx; ++t) {
      const float2 *pl = planes + t * (2 * S * NP) + q0;
#pragma unroll
      for (int r = 0; r < NRX; ++r) {
        const float4 *tl = tb + (r * n_tx + t) * nsel;
        const int *ol = ob + (r * n_tx + t) * nsel;
#pragma unroll KU
        for (int k = 0; k < nsel; ++k) {
          const int ie = (j - it.jf) * NRX * n_tx * nsel + (r * n_tx + t) * nsel + k;
          if (!TT_IN(ie < ck.tap_max && ie < ck.kpad, TT_CHK_TAP_READ)) continue;
          if (!TT_IN(q0 + ol[k] >= 0 && q0 + ol[k] + (S - 1) * NP < 2 * S * NP, TT_CHK_PLANE_READ)) continue;
          const float2 *px = pl + ol[k];
          const float4 h = tl[k];
          const float2 h0 = make_float2(h.x, h.y), dh = make_float2(h.z, h.w);
#pragma unroll
          for (int jj = 0; jj < S; ++jj) {
            const float2 xv = px[jj * NP];
            const float2 hv = tt_fma2(tau2[jj], dh, h0);
            acc[r][jj].x = fmaf(hv.x, xv.x, acc[r][jj].x);
            acc[r][jj].x = fmaf(-hv.y, xv.y, acc[r][jj].x);
            acc[r][jj].y = fmaf(hv.x, xv.y, acc[r][jj].y);
            acc[r][jj].y = fmaf(hv.y, xv.x, acc[r][jj].y);
          }
        }
      }
    }
  } else {
  const float4 *tb = taps + (j - it.jf) * per;
  for (int t = 0; t < n_tx; ++t) {
    const float2 *pl = planes + t * (2 * S * NP) + q0;
    const float4 *tbt = tb + t * K;
#pragma unroll KU
    for (int k = 0; k < K; ++k) {
      if (!TT_IN(k < ck.kpad && (j - it.jf) * per + (NRX - 1) * n_tx * K + t * K + k < ck.tap_max,
                 TT_CHK_TAP_READ))
        continue;
      if (!TT_IN(q0 + offk[k] >= 0 && q0 + offk[k] + (S - 1) * NP < 2 * S * NP, TT_CHK_PLANE_READ)) continue;
      const float2 *px = pl + offk[k];
      float2 xv[S];
#pragma unroll
      for (int jj = 0; jj < S; ++jj) xv[jj] = px[jj * NP];
#pragma unroll
      for (int r = 0; r < NRX; ++r) {
        const float4 h = tbt[r * n_tx * K + k];
        const float2 h0 = make_float2(h.x, h.y), dh = make_float2(h.z, h.w);
#pragma unroll
        for (int jj = 0; jj < S; ++jj) {
          const float2 hv = tt_fma2(tau2[jj], dh, h0);  // h(m) = H[a] + tau (H[a+1] - H[a])
          acc[r][jj].x = fmaf(hv.x, xv[jj].x, acc[r][jj].x);
          acc[r][jj].x = fmaf(-hv.y, xv[jj].y, acc[r][jj].x);
          acc[r][jj].y = fmaf(hv.x, xv[jj].y, acc[r][jj].y);
          acc[r][jj].y = fmaf(hv.y, xv[jj].x, acc[r][jj].y);
        }
      }
    }
  }
  }

  const float nstd = U->noise_std;
  const uint64_t m0 = it.slot * (uint64_t)n + (uint64_t)w_me;
  const int slot_pos = it.slot_pos;
#pragma unroll
  for (int r = 0; r < NRX; ++r) {
    if (nstd > 0.f) {
      if (S == 1) {
        tt_awgn_add_one(U->seed, U->ue_id, (uint32_t)r, m0, nstd, acc[r][0]);
      } else {
#pragma unroll
        for (int jj = 0; jj < S; jj += 2)
          tt_awgn_add_pair(U->seed, U->ue_id, (uint32_t)r, m0 + (uint64_t)jj, nstd, acc[r][jj], acc[r][jj + 1]);
      }
    }
    if (!TT_IN(slot_pos >= 0 && (int64_t)(slot_pos * NRX + r) * n + w_me + S <=
                   (int64_t)U->ring_q * NRX * n - ck.shrink,
               TT_CHK_RING_OUT))
      continue;
    if (U->out_f32) {
      float2 *dstf = reinterpret_cast<float2 *>(U->ring_out) + ((size_t)(slot_pos * NRX + r) * n + w_me);
      if (S >= 2 && (reinterpret_cast<uintptr_t>(dstf) & 15) == 0) {
#pragma unroll
        for (int jj = 0; jj < S; jj += 2)
          *reinterpret_cast<float4 *>(dstf + jj) =
              make_float4(acc[r][jj].x, acc[r][jj].y, acc[r][jj + 1].x, acc[r][jj + 1].y);
      } else {
#pragma unroll
        for (int jj = 0; jj < S; ++jj) dstf[jj] = acc[r][jj];
      }
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

// Single-antenna variants with up to 4 samples per thread fit 64 registers, so eight 128-thread CTAs
// share an SM and hide each other's staging barriers.  At 8 samples per thread 64 registers spill;
// five CTAs (up to 102 registers) ran the 256-UE mixed batch 5% faster than eight and 1% faster
// than six.  At 16 samples per thread, shared memory admits four (48 KB each at delays up to 256),
// and 128 registers hold the variant without spills.  256-thread CTAs ask for half as many, so the
// registers per thread stay the same.  The multi-antenna variants keep the compiler's choice.
constexpr int tt_min_blocks_128(int S, int NRX) {
  return NRX != 1 ? 1 : (S <= 4 ? 8 : (S == 8 ? 5 : 4));
}
constexpr int tt_min_blocks(int S, int NRX, int TPB) {
  return tt_min_blocks_128(S, NRX) * TT_TPB / TPB > 0 ? tt_min_blocks_128(S, NRX) * TT_TPB / TPB : 1;
}

template <int S, int NRX, int DMAX, bool TOPN, int TPB>
__global__ void __launch_bounds__(TPB, tt_min_blocks(S, NRX, TPB))
    tt_conv_fp32_kernel(const TTUEDesc *__restrict__ ues, const TTSeg *__restrict__ segs, int n_segs,
                        uint32_t total_items, uint32_t *__restrict__ counter, int ntx, int tap_max, int k_max,
                        const unsigned long long *__restrict__ cursors, TTCheck ck) {
  constexpr int NP = tt_geo_np(TPB, S, DMAX);
  constexpr int WMAX = tt_geo_wmax(TPB, S, DMAX);
  extern __shared__ float4 dyn_smem[];
  __shared__ TTItem s_it[2];
  __shared__ uint32_t s_claim;
  __shared__ int s_sym[2][TT_MAX_SYM + 1];

  const int tid = threadIdx.x;
  const int kpad = (k_max + 3) & ~3;
  ck.tap_max = tap_max;
  ck.kpad = kpad;
  float2 *planes = reinterpret_cast<float2 *>(dyn_smem);
  uint32_t *raw = reinterpret_cast<uint32_t *>(planes + ntx * 2 * S * NP);
  float4 *taps0 = reinterpret_cast<float4 *>(raw + ((ntx * WMAX + 3) & ~3));
  float4 *taps1 = taps0 + tap_max;
  int *dly0 = reinterpret_cast<int *>(taps1 + tap_max);
  int *dly1 = dly0 + kpad;

  uint32_t next_static = blockIdx.x;
  auto claim = [&]() -> uint32_t {
    if (counter) return atomicAdd(counter, 1u);
    const uint32_t v = next_static;
    next_static += gridDim.x;
    return v;
  };

  // ---- prologue: first item fully staged, second item located ----
  if (tid == 0) {
    tt_locate<TPB>(ues, segs, n_segs, claim(), total_items, cursors, s_it[0]);
    s_claim = claim();
  }
  __syncthreads();
  if (!s_it[0].valid) return;
  {
    const TTItem it = s_it[0];
    const TTUEDesc *U = ues + it.ue;
    tt_issue_item<S, NRX, TOPN, TPB>(U, it, raw, WMAX, taps0, dly0, s_sym[0], tid, ck);
    tt_cp_async_wait_all();
    __syncthreads();
    tt_convert_item<S, NRX, NP, TOPN, WMAX, TPB>(U, it, raw, WMAX, planes, taps0, dly0, tid, ck);
    if (tid == 0) tt_locate<TPB>(ues, segs, n_segs, s_claim, total_items, cursors, s_it[1]);
    __syncthreads();
  }

  int cb = 0;
  for (;;) {
    const TTItem cur = s_it[cb];
    const TTItem nxt = s_it[cb ^ 1];
    float4 *tc = cb ? taps1 : taps0, *tn = cb ? taps0 : taps1;
    int *dc = cb ? dly1 : dly0, *dn = cb ? dly0 : dly1;
    const TTUEDesc *Un = ues + nxt.ue;
    if (nxt.valid) tt_issue_item<S, NRX, TOPN, TPB>(Un, nxt, raw, WMAX, tn, dn, s_sym[cb ^ 1], tid, ck);
    tt_compute_item<S, NRX, NP, TOPN>(ues + cur.ue, cur, planes, tc, dc, s_sym[cb], tid, ck);
    // claimed after the arithmetic: claiming before it measured 4.5% slower on the 16-UE step
    uint32_t nn = 0;
    if (tid == 0 && nxt.valid) nn = claim();
    tt_cp_async_wait_all();
    __syncthreads();
    if (!nxt.valid) return;
    tt_convert_item<S, NRX, NP, TOPN, WMAX, TPB>(Un, nxt, raw, WMAX, planes, tn, dn, tid, ck);
    if (tid == 0) tt_locate<TPB>(ues, segs, n_segs, nn, total_items, cursors, s_it[cb]);
    __syncthreads();
    cb ^= 1;
  }
}

template <int S, int NRX, int DMAX, bool TOPN, int TPB>
cudaError_t tt_launch_variant(const TTLaunch &L, cudaStream_t st) {
  auto kern = tt_conv_fp32_kernel<S, NRX, DMAX, TOPN, TPB>;
  static bool attr_done = false;  // benign race: the attribute call is idempotent
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (L.grid < 0) {  // occupancy query: blocks per SM returned through grid
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, TPB, L.smem) != cudaSuccess) blocks = 1;
    const_cast<TTLaunch &>(L).grid = -(blocks > 0 ? blocks : 1);
    return cudaSuccess;
  }
  if (L.grid == 0 || L.total_items == 0) return cudaSuccess;
  kern<<<L.grid, TPB, L.smem, st>>>(L.ues, L.segs, L.n_segs, L.total_items, L.counter, L.ntx, L.tap_max,
                                    L.k_max, L.cursors, L.check);
  return cudaGetLastError();
}

template <int S, int NRX, bool TOPN, int TPB>
cudaError_t tt_launch_dclass(const TTLaunch &L, cudaStream_t st) {
  switch (L.dclass) {
    case 0: return tt_launch_variant<S, NRX, TT_DCLASS0, TOPN, TPB>(L, st);
    case 1: return tt_launch_variant<S, NRX, TT_DCLASS1, TOPN, TPB>(L, st);
    case 2: return tt_launch_variant<S, NRX, TT_DCLASS2, TOPN, TPB>(L, st);
    case 3: return tt_launch_variant<S, NRX, TT_DCLASS3, TOPN, TPB>(L, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int S, bool TOPN, int TPB>
cudaError_t tt_launch_spt(const TTLaunch &L, cudaStream_t st) {
  if (L.tpb != TPB) return cudaErrorInvalidValue;
  switch (L.nrx) {
    case 1: return tt_launch_dclass<S, 1, TOPN, TPB>(L, st);
    case 2: return tt_launch_dclass<S, 2, TOPN, TPB>(L, st);
    case 3:
      if constexpr (S <= 8) return tt_launch_dclass<S, 3, TOPN, TPB>(L, st);
      return cudaErrorInvalidValue;
    case 4:
      if constexpr (S <= 8) return tt_launch_dclass<S, 4, TOPN, TPB>(L, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tt
