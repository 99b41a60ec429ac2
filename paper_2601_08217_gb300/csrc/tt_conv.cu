// Launch dispatch for the tiled FP32 kernel, its shared-memory sizing, and the
// plain comparison form (one launch per UE per slot, one thread per output
// sample, taps and input read straight from global memory).
#include "tt_conv_kernel.cuh"
#include "tt_internal.h"
#include "tt_philox.cuh"

size_t tt_conv_smem_bytes(int spt, int tpb, int dclass, int n_tx, int tap_max, int k_max) {
  const int dmax = tt_dclass_max(dclass);
  const int np = tt_geo_np(tpb, spt, dmax);
  const int wmax = tt_geo_wmax(tpb, spt, dmax);
  const size_t planes = (size_t)n_tx * 2 * spt * np * sizeof(float2);
  const size_t raw = (size_t)((n_tx * wmax + 3) & ~3) * sizeof(uint32_t);
  const size_t taps = 2 * (size_t)tap_max * sizeof(float4);
  const size_t dly = 2 * (size_t)((k_max + 3) & ~3) * sizeof(int);
  return planes + raw + taps + dly;
}

// For each work item (tpb groups of spt samples) of a slot: first symbol it
// touches and how many symbols it touches, packed as jf | (nst << 16).
int tt_conv_chunk_info(int spt, int tpb, const int32_t *sym_len, int nsym, int32_t *out, int max_out) {
  int n = 0;
  for (int j = 0; j < nsym; ++j) n += sym_len[j];
  const int groups = n / spt;
  const int items = (groups + tpb - 1) / tpb;
  if (items > max_out) return -1;
  for (int c = 0; c < items; ++c) {
    const int g0 = c * tpb;
    const int w0 = g0 * spt;
    const int wl = (g0 + tpb < groups ? g0 + tpb : groups) * spt - 1;
    int b = 0, j0 = -1, j1 = -1;
    for (int j = 0; j < nsym; ++j) {
      if (j0 < 0 && w0 < b + sym_len[j]) j0 = j;
      if (j1 < 0 && wl < b + sym_len[j]) j1 = j;
      b += sym_len[j];
    }
    out[c] = j0 | ((j1 - j0 + 1) << 16);
  }
  return items;
}

int tt_checked_build() {
#if defined(TT_CHECKED) && TT_CHECKED
  return 1;
#else
  return 0;
#endif
}

cudaError_t tt_launch_conv_fp32(const TTLaunch &L, cudaStream_t st) {
  const bool w = L.tpb == TT_TPB_WIDE;
  if (!w && L.tpb != TT_TPB) return cudaErrorInvalidValue;
  if (L.topn) {
    switch (L.spt) {
      case 1: return w ? tt_launch_conv_s1_w_topn(L, st) : tt_launch_conv_s1_topn(L, st);
      case 2: return w ? tt_launch_conv_s2_w_topn(L, st) : tt_launch_conv_s2_topn(L, st);
      case 4: return w ? tt_launch_conv_s4_w_topn(L, st) : tt_launch_conv_s4_topn(L, st);
      case 8: return w ? tt_launch_conv_s8_w_topn(L, st) : tt_launch_conv_s8_topn(L, st);
      case 16: return w ? tt_launch_conv_s16_w_topn(L, st) : tt_launch_conv_s16_topn(L, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.spt) {
    case 1: return w ? tt_launch_conv_s1_w(L, st) : tt_launch_conv_s1(L, st);
    case 2: return w ? tt_launch_conv_s2_w(L, st) : tt_launch_conv_s2(L, st);
    case 4: return w ? tt_launch_conv_s4_w(L, st) : tt_launch_conv_s4(L, st);
    case 8: return w ? tt_launch_conv_s8_w(L, st) : tt_launch_conv_s8(L, st);
    case 16: return w ? tt_launch_conv_s16_w(L, st) : tt_launch_conv_s16(L, st);
    default: return cudaErrorInvalidValue;
  }
}

// Device-resident slot cursors: after a graph replay every run advances by its slot count times
// the number of lanes the replays rotate over (a lane's next replay is that many steps later).
__global__ void tt_advance_kernel(const TTSeg *__restrict__ segs, int n_segs, unsigned long long *cursors,
                                  unsigned stride) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_segs) cursors[segs[i].ue] += (unsigned long long)segs[i].n_slots * stride;
}

cudaError_t tt_launch_advance(const TTSeg *segs, int n_segs, unsigned long long *cursors, unsigned stride,
                              cudaStream_t st) {
  if (n_segs <= 0) return cudaSuccess;
  tt_advance_kernel<<<(n_segs + 127) / 128, 128, 0, st>>>(segs, n_segs, cursors, stride);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plain form: the straightforward mapping, kept as the comparison point.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tt_plain_kernel(const TTUEDesc *__restrict__ U, uint64_t slot) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = U->n;
  if (w >= n) return;
  const int nsym = U->nsym, n_tx = U->n_tx, n_rx = U->n_rx, K = U->n_taps, Q = U->ring_q;
  int j = 0;
  while (j + 1 < nsym && U->sym_start[j + 1] <= w) ++j;
  const float tau = (float)(w - U->sym_start[j]) / (float)(U->sym_start[j + 1] - U->sym_start[j]);
  const uint64_t a = slot * (uint64_t)nsym + (uint64_t)j;
  const int per = n_rx * n_tx * K;
  const int slot_pos = (int)(slot % (uint64_t)Q);
  const uint32_t *rin = reinterpret_cast<const uint32_t *>(U->ring_in);
  const uint64_t m = slot * (uint64_t)n + (uint64_t)w;
  for (int r = 0; r < n_rx; ++r) {
    float yr = 0.f, yi = 0.f;
    for (int t = 0; t < n_tx; ++t) {
      for (int k = 0; k < K; ++k) {
        const int e = (r * n_tx + t) * K + k;
        const float2 h0 = tt::tt_anchor(U, a, e, per);
        const float2 h1 = tt::tt_anchor(U, a + 1, e, per);
        const float hr = fmaf(tau, h1.x - h0.x, h0.x);
        const float hi = fmaf(tau, h1.y - h0.y, h0.y);
        int src = w - U->delays[k];
        int pos = slot_pos;
        if (src < 0) {
          const int back = (-src + n - 1) / n;
          src += back * n;
          pos -= back;
          while (pos < 0) pos += Q;
        }
        const float2 x = tt_unpack_iq(rin[(size_t)(pos * n_tx + t) * n + src]);
        yr = fmaf(hr, x.x, yr);
        yr = fmaf(-hi, x.y, yr);
        yi = fmaf(hr, x.y, yi);
        yi = fmaf(hi, x.x, yi);
      }
    }
    if (U->noise_std > 0.f) {
      const float2 z = tt_awgn_one(U->seed, U->ue_id, (uint32_t)r, m);
      yr = fmaf(U->noise_std, z.x, yr);
      yi = fmaf(U->noise_std, z.y, yi);
    }
    const size_t o = (size_t)(slot_pos * n_rx + r) * n + w;
    if (U->out_f32)
      reinterpret_cast<float2 *>(U->ring_out)[o] = make_float2(yr, yi);
    else
      reinterpret_cast<uint32_t *>(U->ring_out)[o] = tt_pack_iq(yr, yi);
  }
}

// Completion stamp of a batch: the device's global nanosecond timer, written by one thread after
// every earlier kernel of the stream has finished.
__global__ void tt_stamp_kernel(unsigned long long *dst) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *dst = t;
}

cudaError_t tt_launch_stamp(unsigned long long *dst, cudaStream_t st) {
  tt_stamp_kernel<<<1, 1, 0, st>>>(dst);
  return cudaGetLastError();
}

cudaError_t tt_launch_plain(const TTUEDesc *ue_dev, uint64_t slot, int n, cudaStream_t st) {
  const int tpb = 256;
  tt_plain_kernel<<<(n + tpb - 1) / tpb, tpb, 0, st>>>(ue_dev, slot);
  return cudaGetLastError();
}

// ---- uplink aggregation at a cell: one thread per (slot, Rx antenna, pair of samples) ----
__global__ void __launch_bounds__(256) tt_cell_reduce_kernel(TTCellArgs A, uint64_t first_slot) {
  const int pairs = A.n >> 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.n_rx * pairs) return;
  const uint64_t s = first_slot + blockIdx.y;
  const int r = idx / pairs, m = 2 * (idx - r * pairs);
  float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
  for (int u = 0; u < A.n_members; ++u) {  // member order: the FP32 sums are reproducible
    const TTCellMember mb = A.members[u];
    const float4 v = *reinterpret_cast<const float4 *>(
        mb.ring_out + ((size_t)(s % (uint64_t)mb.ring_q) * A.n_rx + r) * A.n + m);
    y0.x += v.x;
    y0.y += v.y;
    y1.x += v.z;
    y1.y += v.w;
  }
  if (A.noise_std > 0.f) tt_awgn_add_pair(A.seed, A.cell_id, (uint32_t)r, s * (uint64_t)A.n + (uint64_t)m, A.noise_std, y0, y1);
  const size_t o = ((size_t)(s % (uint64_t)A.ring_q) * A.n_rx + r) * A.n + m;
  if (A.out_f32) {
    *reinterpret_cast<float4 *>(reinterpret_cast<float2 *>(A.ring_out) + o) = make_float4(y0.x, y0.y, y1.x, y1.y);
  } else {
    *reinterpret_cast<uint2 *>(reinterpret_cast<uint32_t *>(A.ring_out) + o) =
        make_uint2(tt_pack_iq(y0.x, y0.y), tt_pack_iq(y1.x, y1.y));
  }
}

cudaError_t tt_launch_cell_reduce(const TTCellArgs &A, uint64_t first_slot, uint32_t n_slots, cudaStream_t st) {
  if (n_slots == 0) return cudaSuccess;
  const int tpb = 256, work = A.n_rx * (A.n >> 1);
  tt_cell_reduce_kernel<<<dim3((work + tpb - 1) / tpb, n_slots), tpb, 0, st>>>(A, first_slot);
  return cudaGetLastError();
}

// ---- continuous CIR resampled onto the fixed delay grid: one thread per (step, link, tap) ----
// Band-limited discrete-time equivalent of the multipath channel: the tap at delay k is the sum of
// the paths' gains weighted by sinc(k - tau_p), tau_p the path delay in samples; FP64 throughout.
__global__ void tt_cir_resample_kernel(const float2 *__restrict__ gains, const double *__restrict__ tau, int n_steps,
                                       int n_links, int n_paths, int n_taps, float2 *__restrict__ taps) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)n_steps * n_links * n_taps;
  if (idx >= total) return;
  const int k = (int)(idx % n_taps);
  const long long tl = idx / n_taps;  // step * n_links + link
  const int t = (int)(tl / n_links);
  double re = 0.0, im = 0.0;
  for (int p = 0; p < n_paths; ++p) {
    const double v = (double)k - tau[(size_t)t * n_paths + p];
    const double s = v == 0.0 ? 1.0 : sinpi(v) / (3.141592653589793 * v);
    const float2 a = gains[(size_t)tl * n_paths + p];
    re += (double)a.x * s;
    im += (double)a.y * s;
  }
  taps[idx] = make_float2((float)re, (float)im);
}

cudaError_t tt_launch_cir_resample(const float2 *gains, const double *tau, int n_steps, int n_links, int n_paths,
                                   int n_taps, float2 *taps, cudaStream_t st) {
  const long long total = (long long)n_steps * n_links * n_taps;
  if (total == 0) return cudaSuccess;
  const int tpb = 256;
  tt_cir_resample_kernel<<<(unsigned)((total + tpb - 1) / tpb), tpb, 0, st>>>(gains, tau, n_steps, n_links, n_paths,
                                                                                n_taps, taps);
  return cudaGetLastError();
}

// ---- sum-of-sinusoids anchors: one thread per (job, slot, link tap) ----
// The phase f t + p at the slot's start is reduced modulo 2 pi in FP64 once per sinusoid; the
// symbols inside the slot add f (b_j - b_0) / f_s (under 2 pi f_D x one slot) in FP32.
__global__ void __launch_bounds__(128) tt_sos_kernel(const TTSosJob *__restrict__ jobs, int n_jobs,
                                                     unsigned long long n_threads) {
  const unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_threads) return;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].thread_begin <= idx) lo = mid; else hi = mid - 1;
  }
  const TTSosJob J = jobs[lo];
  const unsigned long long rel = idx - J.thread_begin;
  const int e = (int)(rel % (unsigned long long)J.per);
  const int sl = (int)(rel / (unsigned long long)J.per);   // 0 .. n_slots (n_slots: the tail anchor)
  const TTUEDesc *U = J.ue;
  const int nsym = U->nsym, n_sym_here = sl < J.n_slots ? nsym : 1;
  const uint64_t s = J.slot_first + (uint64_t)sl;
  const double t0 = (double)(s * (uint64_t)U->n) * J.inv_fs;
  const double two_pi = 6.283185307179586, inv_two_pi = 0.15915494309189535;
  float si[TT_MAX_SYM], sq[TT_MAX_SYM];
#pragma unroll
  for (int j = 0; j < TT_MAX_SYM; ++j) si[j] = sq[j] = 0.f;
  const double *f = J.freq + (size_t)e * J.m * 2, *p = J.phase + (size_t)e * J.m * 2;
  for (int n = 0; n < J.m; ++n) {
    const double ai = fma(f[2 * n], t0, p[2 * n]), aq = fma(f[2 * n + 1], t0, p[2 * n + 1]);
    const float bi = (float)fma(-rint(ai * inv_two_pi), two_pi, ai), bq = (float)fma(-rint(aq * inv_two_pi), two_pi, aq);
    const float fi = (float)(f[2 * n] * J.inv_fs), fq = (float)(f[2 * n + 1] * J.inv_fs);   // rad per sample
#pragma unroll
    for (int j = 0; j < TT_MAX_SYM; ++j) {
      if (j < n_sym_here) {
        const float off = (float)U->sym_start[j];
        si[j] += cosf(fmaf(fi, off, bi));
        sq[j] += cosf(fmaf(fq, off, bq));
      }
    }
  }
  const float g = J.amp[e] * rsqrtf((float)J.m);
  const uint64_t a0 = s * (uint64_t)nsym;
#pragma unroll
  for (int j = 0; j < TT_MAX_SYM; ++j)
    if (j < n_sym_here) J.ring[(size_t)((a0 + (uint64_t)j) % (uint64_t)J.ring_len) * J.per + e] = make_float2(g * si[j], g * sq[j]);
}

cudaError_t tt_launch_sos(const TTSosJob *jobs, int n_jobs, unsigned long long n_threads, cudaStream_t st) {
  if (n_threads == 0 || n_jobs == 0) return cudaSuccess;
  const int tpb = 128;
  tt_sos_kernel<<<(unsigned)((n_threads + tpb - 1) / tpb), tpb, 0, st>>>(jobs, n_jobs, n_threads);
  return cudaGetLastError();
}

// ---- timed traces: per-symbol anchors in FP64 trace time, one warp per (job, anchor) ----
// Lane 0 places the anchor in trace time (FP64: p = b / step, i0 = floor(p), f = p - i0, the same
// steps as the convolution kernels' tt_anchor) and broadcasts it; the lanes interpolate the link
// taps, H = h[i0] + f (h[i0 + 1] - h[i0]) in FP64, coalesced along the taps.
__global__ void __launch_bounds__(128) tt_retime_kernel(const TTRetimeJob *__restrict__ jobs, int n_jobs,
                                                        unsigned long long n_warps) {
  const unsigned long long gw = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= n_warps) return;  // whole warps leave together
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].thread_begin <= gw) lo = mid; else hi = mid - 1;
  }
  const TTRetimeJob J = jobs[lo];
  const TTUEDesc *U = J.ue;
  const uint64_t nsym = (uint64_t)U->nsym;
  const uint64_t a = J.slot_first * nsym + (gw - J.thread_begin);   // the job's anchors, the tail last
  unsigned long long i0 = 0;
  double f = 0.0;
  if (lane == 0) {
    const uint64_t b = (a / nsym) * (uint64_t)U->n + (uint64_t)U->sym_start[a % nsym];
    const double p = (double)b / J.step;
    const double fl = floor(p);
    f = p - fl;
    i0 = (unsigned long long)fl;
  }
  i0 = __shfl_sync(0xFFFFFFFFu, i0, 0);
  f = __shfl_sync(0xFFFFFFFFu, f, 0);
  const uint64_t T = J.T;
  const uint64_t k0 = J.loop ? (i0 % T) : (i0 < T ? i0 : T - 1);
  const uint64_t k1 = J.loop ? ((i0 + 1) % T) : (i0 + 1 < T ? i0 + 1 : T - 1);
  const float2 *h0p = J.src + k0 * (uint64_t)J.per, *h1p = J.src + k1 * (uint64_t)J.per;
  float2 *dst = J.ring + (size_t)(a % (uint64_t)J.ring_len) * J.per;
  for (int e = lane; e < J.per; e += 32) {
    const float2 h0 = __ldg(h0p + e), h1 = __ldg(h1p + e);
    dst[e] = make_float2((float)((double)h0.x + f * ((double)h1.x - (double)h0.x)),
                         (float)((double)h0.y + f * ((double)h1.y - (double)h0.y)));
  }
}

cudaError_t tt_launch_retime(const TTRetimeJob *jobs, int n_jobs, unsigned long long n_warps, cudaStream_t st) {
  if (n_warps == 0 || n_jobs == 0) return cudaSuccess;
  const int tpb = 128;
  tt_retime_kernel<<<(unsigned)((n_warps * 32 + tpb - 1) / tpb), tpb, 0, st>>>(jobs, n_jobs, n_warps);
  return cudaGetLastError();
}

// ---- sparse convolution: per (anchor, link) tap selection, one warp each ----
__global__ void __launch_bounds__(256) tt_topn_select_kernel(const TTTopnJob *__restrict__ jobs, int n_jobs,
                                                             unsigned long long n_warps) {
  const unsigned long long gw = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= n_warps) return;  // whole warps leave together
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].warp_begin <= gw) lo = mid; else hi = mid - 1;
  }
  const TTTopnJob J = jobs[lo];
  const unsigned long long rel = gw - J.warp_begin;
  const int l = (int)(rel % (unsigned long long)J.links);
  const uint64_t a = J.a_first + rel / (unsigned long long)J.links;
  const TTUEDesc *U = J.ue;
  const int K = U->n_taps, nsel = U->top_n, per = J.links * K;
  constexpr int R = TT_MAX_TAPS / 32;  // taps per lane
  float4 hv[R];
  float pw[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int k = lane + 32 * i;
    pw[i] = -1.f;  // below every power: absent taps never beat a present one
    if (k < K) {
      const float2 h0 = tt::tt_anchor(U, a, l * K + k, per), h1 = tt::tt_anchor(U, a + 1, l * K + k, per);
      hv[i] = make_float4(h0.x, h0.y, h1.x - h0.x, h1.y - h0.y);
      pw[i] = __fmaf_rn(h0.x, h0.x, __fmul_rn(h0.y, h0.y));
    }
  }
  // rank of each of this lane's taps: the taps that beat it (higher power, or equal and lower index)
  int beat[R];
#pragma unroll
  for (int i = 0; i < R; ++i) beat[i] = 0;
#pragma unroll
  for (int ji = 0; ji < R; ++ji) {
    if (32 * ji >= K) break;
    for (int jl = 0; jl < 32; ++jl) {
      const int j = 32 * ji + jl;
      const float pj = __shfl_sync(0xFFFFFFFFu, pw[ji], jl);
      if (j < K) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int k = lane + 32 * i;
          beat[i] += (pj > pw[i]) || (pj == pw[i] && j < k);
        }
      }
    }
  }
  // compaction in tap order: position = kept taps of lower index
  const size_t base = (size_t)(a % (uint64_t)U->sparse_len) * (size_t)(J.links * nsel) + (size_t)l * nsel;
  float4 *ring = const_cast<float4 *>(U->sparse);
  int32_t *dring = const_cast<int32_t *>(U->sparse_dly);
  int before = 0;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int k = lane + 32 * i;
    const bool keep = k < K && beat[i] < nsel;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep) {
      const int pos = before + __popc(m & ((1u << lane) - 1u));
      ring[base + pos] = hv[i];
      dring[base + pos] = U->delays[k];
    }
    before += __popc(m);
  }
}

cudaError_t tt_launch_topn_select(const TTTopnJob *jobs, int n_jobs, unsigned long long n_warps, cudaStream_t st) {
  if (n_warps == 0 || n_jobs == 0) return cudaSuccess;
  const unsigned long long threads = n_warps * 32;
  tt_topn_select_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(jobs, n_jobs, n_warps);
  return cudaGetLastError();
}
