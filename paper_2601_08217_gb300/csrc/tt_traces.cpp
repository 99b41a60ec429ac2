// Channel traces: loading a stored, timed or continuous-CIR trace, on-device tap synthesis, and the
// per-run pre-passes that prepare a run's anchors (timed-trace retiming, synthesis, top-n tap
// selection).  Sec. IV (channel traces replayed per UE), Sec. III-C (top-n sparse convolution).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "tt_chan.h"
#include "tt_engine_impl.h"
#include "tt_internal.h"

using ttx::chunk_table;
using ttx::dfree;
using ttx::dmalloc;
using ttx::drop_graph;
using ttx::fail;
using ttx::pick_dclass;
using ttx::set_geom;
using ttx::spt_candidates;
using ttx::sparse;
using ttx::update_chan;
using ttx::update_completed;
using ttx::upload_desc;
using ttx::valid_chan;

namespace {

// Check a trace's delays and geometry against the channel and pick the tiled-kernel geometry
// (engine lock not needed: reads the channel's configuration and the tuning cache only).
struct TraceGeo {
  int d_max = 0, dclass = 0, spt = 0, tpb = TT_TPB, tap_need = 0;
  size_t smem = 0;
};
tt_status trace_geometry(const tt_chan *c, const int32_t *delays, uint32_t n_taps, TraceGeo &g) {
  g.d_max = 0;
  for (uint32_t k = 0; k < n_taps; ++k) {
    const int32_t d = delays[k];
    if (d < 0 || (uint32_t)d > c->cfg.max_delay) return fail(TT_ERR_TRACE, "delay %d outside 0..%u", d, c->cfg.max_delay);
    if (k && d < delays[k - 1]) return fail(TT_ERR_TRACE, "delays must be non-decreasing");
    g.d_max = std::max(g.d_max, (int)d);
  }
  g.dclass = pick_dclass(g.d_max);
  const bool tc = c->cfg.precision != TT_FP32;
  if (tc && g.d_max > tt_tc_max_delay())
    return fail(TT_ERR_TRACE, "tensor-core channels take delays up to %d (got %d)", tt_tc_max_delay(), g.d_max);
  if (tc)
    for (uint32_t v : c->sym_len)
      if (v % 8) return fail(TT_ERR_INVALID, "tensor-core channels need symbol lengths divisible by 8");
  const bool topn = c->cfg.top_n > 0 && c->cfg.top_n < n_taps;
  auto fits = [&](int s, int t) {
    int touched = 1;
    chunk_table(c->sym_len, s, t, &touched);
    const int need = touched * (int)(c->cfg.n_rx * c->cfg.n_tx * n_taps);
    const size_t b = tt_conv_smem_bytes(s, t, g.dclass, c->cfg.n_tx, need, topn ? std::max((int)n_taps, need) : (int)n_taps);
    if (b > 200 * 1024) return false;
    g.spt = s;
    g.tpb = t;
    g.tap_need = need;
    g.smem = b;
    return true;
  };
  // largest samples-per-thread whose shared-memory footprint fits at 128 threads, or at the
  // engine's thread count (the tensor-core form keeps the smallest valid tiled geometry, unused)
  const int tpb = c->e->tpb_override ? (int)c->e->tpb_override : TT_TPB;
  g.spt = 0;
  for (int s : spt_candidates(c->sym_len, c->e->spt_override, c->cfg.n_rx, c->cfg.n_tx)) {
    if (tc) {
      g.spt = 1;
      break;
    }
    if (fits(s, tpb)) break;
  }
  if (g.spt == 0)
    return fail(TT_ERR_INVALID, "channel too large for the tiled kernel: %u x %u antennas, %u taps, delay %d",
                c->cfg.n_rx, c->cfg.n_tx, n_taps, g.d_max);
  // a choice the autotuner made for this class on this device model (TT_TUNE_CACHE) replaces it
  int cs = 0, ct = 0;
  if (!tc && ttx::tune_lookup(c->e, ttx::tune_class_key(c, n_taps, g.dclass), &cs, &ct)) {
    const TraceGeo keep = g;
    const std::vector<int> ok = spt_candidates(c->sym_len, ttx::tune_spt_cap(c->e), c->cfg.n_rx, c->cfg.n_tx);
    const bool count_ok = c->e->tpb_override ? ct == (int)c->e->tpb_override : (ct == TT_TPB || ct == TT_TPB_WIDE);
    if (!count_ok || std::find(ok.begin(), ok.end(), cs) == ok.end() || !fits(cs, ct))
      g = keep;
  }
  return TT_OK;
}

// Replace the channel's trace by device buffers already filled (ownership passes to the channel).
// Engine lock held; no launched work of the channel may be in flight.
tt_status install_trace(tt_chan *c, float2 *taps, int32_t *delays, uint64_t bytes, uint32_t n_anchors,
                        uint32_t n_taps, double step_samples, int loop, const TraceGeo &g) {
  tt_engine *e = c->e;
  // A timed trace stays as it is; the kernels read a ring of per-symbol anchors, sized like the
  // synthesis ring, that a pre-pass refills from it before each run.
  float2 *ring = nullptr;
  uint32_t ring_len = 0;
  if (step_samples > 0.0) {
    ring_len = (uint32_t)((c->Q + 1) * (int)c->sym_len.size() + 1);
    const uint64_t rb = (uint64_t)ring_len * c->cfg.n_rx * c->cfg.n_tx * n_taps * sizeof(float2);
    cudaError_t err = cudaSuccess;
    if (e->budget && e->in_use - c->trace_bytes + bytes + rb > e->budget) {
      err = cudaErrorMemoryAllocation;
    } else {
      err = dmalloc(e, &ring, rb);
      if (err == cudaSuccess) err = cudaMemsetAsync(ring, 0, rb, e->stream);
    }
    if (err != cudaSuccess) {
      dfree(e, ring);
      dfree(e, taps);
      dfree(e, delays);
      return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA,
                  "admission refused or failed: anchor ring of %llu B for the timed trace", (unsigned long long)rb);
    }
    bytes += rb;
  }
  dfree(e, c->d_src);
  c->d_src = nullptr;
  c->retime = false;
  if (ring) {
    c->retime = true;
    c->d_src = taps;
    c->src_T = n_anchors;
    c->src_step = step_samples;
    c->src_loop = loop ? 1 : 0;
    taps = ring;
    n_anchors = ring_len;
    step_samples = 0.0;
    loop = 1;
  }
  dfree(e, c->d_taps);
  dfree(e, c->d_delays);
  dfree(e, c->d_amp);
  dfree(e, c->d_freq);
  dfree(e, c->d_phase);
  c->d_amp = nullptr;
  c->d_freq = c->d_phase = nullptr;
  c->synth = false;
  e->in_use = e->in_use - c->trace_bytes + bytes;
  c->trace_bytes = bytes;
  c->d_taps = taps;
  c->d_delays = delays;
  c->has_trace = true;
  c->dclass = g.dclass;
  c->smem = g.smem;
  c->tap_need = g.tap_need;
  drop_graph(e);
  TTUEDesc &d = c->desc;
  d.taps = taps;
  d.delays = delays;
  d.step_samples = step_samples;
  d.n_taps = (int)n_taps;
  d.d_max = g.d_max;
  d.n_anchors = (int)n_anchors;
  d.loop = loop ? 1 : 0;
  // sparse convolution: a ring of the kept taps per anchor and link, sized like the slot ring
  dfree(e, c->d_sparse);
  dfree(e, c->d_sparse_dly);
  c->d_sparse = nullptr;
  c->d_sparse_dly = nullptr;
  e->in_use -= c->sparse_bytes;
  c->sparse_bytes = 0;
  d.sparse = nullptr;
  d.sparse_dly = nullptr;
  d.sparse_len = 0;
  if (c->cfg.top_n > 0 && c->cfg.top_n < n_taps) {
    const int len = (c->Q + 1) * (int)c->sym_len.size() + 1;
    const size_t ent = (size_t)len * c->cfg.n_rx * c->cfg.n_tx * c->cfg.top_n;
    cudaError_t err = dmalloc(e, &c->d_sparse, ent * sizeof(float4));
    if (err == cudaSuccess) err = dmalloc(e, &c->d_sparse_dly, ent * sizeof(int32_t));
    if (err != cudaSuccess) {
      dfree(e, c->d_sparse);
      c->d_sparse = nullptr;
      c->has_trace = false;
      return fail(TT_ERR_NO_MEMORY, "sparse tap ring: %s", cudaGetErrorString(err));
    }
    c->sparse_bytes = ent * (sizeof(float4) + sizeof(int32_t));
    e->in_use += c->sparse_bytes;
    d.sparse = c->d_sparse;
    d.sparse_dly = c->d_sparse_dly;
    d.sparse_len = len;
  }
  tt_status sst = set_geom(c, g.spt, g.tpb);
  if (sst != TT_OK) return sst;
  if (c->cfg.precision != TT_FP32) {  // the tensor-core kernel's work items: one per symbol
    std::vector<int32_t> L32(c->sym_len.begin(), c->sym_len.end());
    d.items_per_slot = tt_tc_items_per_slot(L32.data(), (int)L32.size());
  }
  return upload_desc(c);
}

// Engine lock held: fail unless the channel has no launched work in flight.
tt_status idle_or_fail(tt_chan *c) {
  tt_engine *e = c->e;
  update_chan(c);
  if (c->launched_end != c->completed_end) {
    cudaError_t q = update_completed(e);
    if (q != cudaSuccess) return fail(TT_ERR_CUDA, "%s", cudaGetErrorString(q));
    update_chan(c);
    if (c->launched_end != c->completed_end) return fail(TT_ERR_STATE, "work in flight; sync first");
  }
  return TT_OK;
}

}  // namespace

tt_status tt_chan_load_trace(tt_chan *c, const tt_trace_desc *tr) {
  if (!valid_chan(c) || !tr || tr->struct_size < sizeof(tt_trace_desc))
    return fail(TT_ERR_INVALID, "tt_chan_load_trace: bad argument");
  tt_engine *e = c->e;
  if (!tr->taps || !tr->delays || tr->n_anchors == 0 || tr->n_taps == 0)
    return fail(TT_ERR_TRACE, "empty trace");
  if (tr->n_taps > c->cfg.max_taps) return fail(TT_ERR_TRACE, "trace has %u taps, max_taps is %u", tr->n_taps,
                                                c->cfg.max_taps);
  if (!(tr->step_samples >= 0.0) || !std::isfinite(tr->step_samples))
    return fail(TT_ERR_TRACE, "bad step_samples");
  TraceGeo g;
  tt_status gs = trace_geometry(c, tr->delays, tr->n_taps, g);
  if (gs != TT_OK) return gs;
  const size_t per = (size_t)c->cfg.n_rx * c->cfg.n_tx * tr->n_taps;
  const size_t nval = per * tr->n_anchors * 2;
  for (size_t i = 0; i < nval; ++i)
    if (!std::isfinite(tr->taps[i])) return fail(TT_ERR_TRACE, "non-finite tap value at %zu", i);

  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status st = idle_or_fail(c);
  if (st != TT_OK) return st;
  const uint64_t bytes = nval * sizeof(float) + tr->n_taps * sizeof(int32_t);
  if (e->budget && e->in_use - c->trace_bytes + bytes > e->budget)
    return fail(TT_ERR_NO_MEMORY, "admission refused: trace of %llu B does not fit the budget",
                (unsigned long long)bytes);
  TT_CK(cudaStreamSynchronize(e->stream));
  float2 *taps = nullptr;
  int32_t *delays = nullptr;
  cudaError_t err = dmalloc(c->e, &taps, nval * sizeof(float));
  if (err == cudaSuccess) err = dmalloc(c->e, &delays, tr->n_taps * sizeof(int32_t));
  if (err == cudaSuccess) err = cudaMemcpy(taps, tr->taps, nval * sizeof(float), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(delays, tr->delays, tr->n_taps * sizeof(int32_t), cudaMemcpyHostToDevice);
  // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
  // streams are not ordered after the default stream: let them land before any kernel reads them
  if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
  if (err != cudaSuccess) {
    dfree(c->e, taps);
    dfree(c->e, delays);
    return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA, "trace upload: %s",
                cudaGetErrorString(err));
  }
  return install_trace(c, taps, delays, bytes, tr->n_anchors, tr->n_taps, tr->step_samples, tr->loop, g);
}

tt_status tt_chan_load_jakes(tt_chan *c, const tt_jakes_desc *j) {
  if (!valid_chan(c) || !j || j->struct_size < sizeof(tt_jakes_desc))
    return fail(TT_ERR_INVALID, "tt_chan_load_jakes: bad argument");
  tt_engine *e = c->e;
  if (!j->delays || !j->amplitude || !j->freq || !j->phase || j->n_taps == 0) return fail(TT_ERR_TRACE, "empty model");
  if (j->n_sinusoids < 1 || j->n_sinusoids > 64) return fail(TT_ERR_TRACE, "n_sinusoids must be 1..64");
  if (j->n_taps > c->cfg.max_taps) return fail(TT_ERR_TRACE, "%u taps, max_taps is %u", j->n_taps, c->cfg.max_taps);
  if (!(j->sample_rate_hz > 0.0) || !std::isfinite(j->sample_rate_hz)) return fail(TT_ERR_TRACE, "bad sample_rate_hz");
  const size_t per = (size_t)c->cfg.n_rx * c->cfg.n_tx * j->n_taps, nfp = per * j->n_sinusoids * 2;
  for (size_t i = 0; i < per; ++i)
    if (!std::isfinite(j->amplitude[i])) return fail(TT_ERR_TRACE, "non-finite amplitude at %zu", i);
  for (size_t i = 0; i < nfp; ++i)
    if (!std::isfinite(j->freq[i]) || !std::isfinite(j->phase[i])) return fail(TT_ERR_TRACE, "non-finite sinusoid at %zu", i);
  TraceGeo g;
  tt_status gs = trace_geometry(c, j->delays, j->n_taps, g);
  if (gs != TT_OK) return gs;

  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status st = idle_or_fail(c);
  if (st != TT_OK) return st;
  // anchor ring: every slot the channel's rings can hold, plus the anchor after the last one
  const uint32_t ring_len = (uint32_t)((c->Q + 1) * (int)c->sym_len.size() + 1);
  const uint64_t bytes = (uint64_t)ring_len * per * sizeof(float2) + j->n_taps * sizeof(int32_t) +
                         per * sizeof(float) + nfp * 2 * sizeof(double);
  if (e->budget && e->in_use - c->trace_bytes + bytes > e->budget)
    return fail(TT_ERR_NO_MEMORY, "admission refused: model of %llu B does not fit the budget", (unsigned long long)bytes);
  TT_CK(cudaStreamSynchronize(e->stream));
  float2 *taps = nullptr;
  int32_t *delays = nullptr;
  float *amp = nullptr;
  double *freq = nullptr, *phase = nullptr;
  cudaError_t err = dmalloc(c->e, &taps, (size_t)ring_len * per * sizeof(float2));
  if (err == cudaSuccess) err = dmalloc(c->e, &delays, j->n_taps * sizeof(int32_t));
  if (err == cudaSuccess) err = dmalloc(c->e, &amp, per * sizeof(float));
  if (err == cudaSuccess) err = dmalloc(c->e, &freq, nfp * sizeof(double));
  if (err == cudaSuccess) err = dmalloc(c->e, &phase, nfp * sizeof(double));
  if (err == cudaSuccess) err = cudaMemcpy(delays, j->delays, j->n_taps * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(amp, j->amplitude, per * sizeof(float), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(freq, j->freq, nfp * sizeof(double), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(phase, j->phase, nfp * sizeof(double), cudaMemcpyHostToDevice);
  // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
  // streams are not ordered after the default stream: let them land before any kernel reads them
  if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
  if (err != cudaSuccess) {
    dfree(c->e, taps);
    dfree(c->e, delays);
    dfree(c->e, amp);
    dfree(c->e, freq);
    dfree(c->e, phase);
    return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA, "model upload: %s", cudaGetErrorString(err));
  }
  st = install_trace(c, taps, delays, bytes, ring_len, j->n_taps, 0.0, 1, g);
  if (st != TT_OK) return st;
  c->synth = true;
  c->d_amp = amp;
  c->d_freq = freq;
  c->d_phase = phase;
  c->synth_m = (int)j->n_sinusoids;
  c->synth_fs = j->sample_rate_hz;
  return TT_OK;
}

tt_status tt_chan_load_cir(tt_chan *c, const tt_cir_desc *cir) {
  if (!valid_chan(c) || !cir || cir->struct_size < sizeof(tt_cir_desc))
    return fail(TT_ERR_INVALID, "tt_chan_load_cir: bad argument");
  tt_engine *e = c->e;
  if (!cir->gains || !cir->delays || cir->n_steps == 0 || cir->n_paths == 0 || cir->n_taps == 0)
    return fail(TT_ERR_TRACE, "empty CIR");
  if (cir->n_taps > c->cfg.max_taps) return fail(TT_ERR_TRACE, "grid of %u taps, max_taps is %u", cir->n_taps,
                                                 c->cfg.max_taps);
  if (!(cir->step_samples >= 0.0) || !std::isfinite(cir->step_samples)) return fail(TT_ERR_TRACE, "bad step_samples");
  const int n_links = (int)(c->cfg.n_rx * c->cfg.n_tx);
  const size_t ng = (size_t)cir->n_steps * n_links * cir->n_paths * 2, nd = (size_t)cir->n_steps * cir->n_paths;
  for (size_t i = 0; i < ng; ++i)
    if (!std::isfinite(cir->gains[i])) return fail(TT_ERR_TRACE, "non-finite path gain at %zu", i);
  for (size_t i = 0; i < nd; ++i)
    if (!std::isfinite(cir->delays[i]) || cir->delays[i] < 0.0) return fail(TT_ERR_TRACE, "bad path delay at %zu", i);
  std::vector<int32_t> grid(cir->n_taps);
  for (uint32_t k = 0; k < cir->n_taps; ++k) grid[k] = (int32_t)k;
  TraceGeo g;
  tt_status gs = trace_geometry(c, grid.data(), cir->n_taps, g);
  if (gs != TT_OK) return gs;

  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  tt_status st = idle_or_fail(c);
  if (st != TT_OK) return st;
  const size_t nval = (size_t)cir->n_steps * n_links * cir->n_taps;
  const uint64_t bytes = nval * sizeof(float2) + cir->n_taps * sizeof(int32_t);
  if (e->budget && e->in_use - c->trace_bytes + bytes > e->budget)
    return fail(TT_ERR_NO_MEMORY, "admission refused: trace of %llu B does not fit the budget",
                (unsigned long long)bytes);
  TT_CK(cudaStreamSynchronize(e->stream));
  float2 *taps = nullptr, *d_gains = nullptr;
  int32_t *delays = nullptr;
  double *d_tau = nullptr;
  cudaError_t err = dmalloc(c->e, &taps, nval * sizeof(float2));
  if (err == cudaSuccess) err = dmalloc(c->e, &delays, cir->n_taps * sizeof(int32_t));
  if (err == cudaSuccess) err = dmalloc(c->e, &d_gains, ng * sizeof(float));
  if (err == cudaSuccess) err = dmalloc(c->e, &d_tau, nd * sizeof(double));
  if (err == cudaSuccess) err = cudaMemcpy(delays, grid.data(), cir->n_taps * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(d_gains, cir->gains, ng * sizeof(float), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(d_tau, cir->delays, nd * sizeof(double), cudaMemcpyHostToDevice);
  // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
  // streams are not ordered after the default stream: let them land before any kernel reads them
  if (err == cudaSuccess) err = cudaStreamSynchronize(nullptr);
  if (err == cudaSuccess)
    err = tt_launch_cir_resample(d_gains, d_tau, (int)cir->n_steps, n_links, (int)cir->n_paths, (int)cir->n_taps,
                                 taps, e->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
  dfree(c->e, d_gains);
  dfree(c->e, d_tau);
  if (err != cudaSuccess) {
    dfree(c->e, taps);
    dfree(c->e, delays);
    return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA, "CIR resampling: %s",
                cudaGetErrorString(err));
  }
  return install_trace(c, taps, delays, bytes, cir->n_steps, cir->n_taps, cir->step_samples, cir->loop, g);
}

namespace ttx {

// Timed traces: refill the anchor rings for the slots this run launches (every symbol of slots
// [launched_end, pushed_end) and the first anchor of slot pushed_end) by FP64 trace-time
// interpolation of the stored trace, all channels in one launch (engine lock held).
tt_status launch_retime(tt_engine *e, const std::vector<tt_chan *> &chans) {
  std::vector<TTRetimeJob> &jobs = e->retime_jobs;
  jobs.clear();
  unsigned long long threads = 0;
  for (tt_chan *c : chans) {
    if (!c->retime || c->pushed_end <= c->launched_end) continue;
    TTRetimeJob J{};
    J.ue = e->d_ues + c->index;
    J.ring = c->d_taps;
    J.src = c->d_src;
    J.step = c->src_step;
    J.T = c->src_T;
    J.loop = c->src_loop;
    J.slot_first = c->launched_end;
    J.thread_begin = threads;
    J.per = (int)(c->cfg.n_rx * c->cfg.n_tx * (uint32_t)c->desc.n_taps);
    J.ring_len = c->desc.n_anchors;
    J.n_slots = (int)(c->pushed_end - c->launched_end);
    threads += (unsigned long long)J.n_slots * c->sym_len.size() + 1;   // one warp per anchor
    jobs.push_back(J);
  }
  if (jobs.empty()) return TT_OK;
  if (jobs.size() > e->retime_cap) {
    TT_CK(cudaStreamSynchronize(e->stream));  // the old list may still be read
    dfree(e, e->d_retime);
    e->d_retime = nullptr;
    e->retime_cap = 0;
    TT_CK(dmalloc(e, &e->d_retime, sizeof(TTRetimeJob) * jobs.size() * 2));
    e->retime_cap = jobs.size() * 2;
  }
  TT_CK(cudaMemcpyAsync(e->d_retime, jobs.data(), sizeof(TTRetimeJob) * jobs.size(), cudaMemcpyHostToDevice,
                        e->stream));
  cudaError_t err = tt_launch_retime(e->d_retime, (int)jobs.size(), threads, e->stream);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "timed-trace anchor launch: %s", cudaGetErrorString(err));
  ++e->launches;
  return TT_OK;
}

// Synthesised channels: fill the anchor rings for the slots this run launches (same anchors as
// above), all channels in one launch (engine lock held).  An anchor rewritten here gets the value it
// had; a position that held an earlier anchor is rewritten only after every batch that read it (the
// engine stream waits for those on other launch lanes before the pre-passes).
tt_status launch_synth(tt_engine *e, const std::vector<tt_chan *> &chans) {
  std::vector<TTSosJob> &jobs = e->sos_jobs;
  jobs.clear();
  unsigned long long threads = 0;
  for (tt_chan *c : chans) {
    if (!c->synth || c->pushed_end <= c->launched_end) continue;
    TTSosJob J{};
    J.ue = e->d_ues + c->index;
    J.ring = c->d_taps;
    J.amp = c->d_amp;
    J.freq = c->d_freq;
    J.phase = c->d_phase;
    J.inv_fs = 1.0 / c->synth_fs;
    J.slot_first = c->launched_end;
    J.thread_begin = threads;
    J.per = (int)(c->cfg.n_rx * c->cfg.n_tx * (uint32_t)c->desc.n_taps);
    J.m = c->synth_m;
    J.ring_len = c->desc.n_anchors;
    J.n_slots = (int)(c->pushed_end - c->launched_end);
    J.tail = 1;
    threads += (unsigned long long)(J.n_slots + 1) * (unsigned long long)J.per;
    jobs.push_back(J);
  }
  if (jobs.empty()) return TT_OK;
  if (jobs.size() > e->sos_cap) {
    TT_CK(cudaStreamSynchronize(e->stream));  // the old list may still be read
    dfree(e, e->d_sos);
    e->d_sos = nullptr;
    e->sos_cap = 0;
    TT_CK(dmalloc(e, &e->d_sos, sizeof(TTSosJob) * jobs.size() * 2));
    e->sos_cap = jobs.size() * 2;
  }
  TT_CK(cudaMemcpyAsync(e->d_sos, jobs.data(), sizeof(TTSosJob) * jobs.size(), cudaMemcpyHostToDevice, e->stream));
  cudaError_t err = tt_launch_sos(e->d_sos, (int)jobs.size(), threads, e->stream);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "synthesis launch: %s", cudaGetErrorString(err));
  ++e->launches;
  return TT_OK;
}

// Sparse convolution: select the kept taps of every anchor this run's slots use (one launch for all
// channels), after any synthesis of the anchors themselves (engine lock held).
tt_status launch_topn(tt_engine *e, const std::vector<tt_chan *> &chans) {
  std::vector<TTTopnJob> &jobs = e->topn_jobs;
  jobs.clear();
  unsigned long long warps = 0;
  for (tt_chan *c : chans) {
    if (!sparse(c) || !c->d_sparse || c->pushed_end <= c->launched_end) continue;
    const uint64_t nsym = c->sym_len.size();
    TTTopnJob J{};
    J.ue = e->d_ues + c->index;
    J.a_first = c->launched_end * nsym;
    J.n_anchors = (int)((c->pushed_end - c->launched_end) * nsym);
    J.links = (int)(c->cfg.n_rx * c->cfg.n_tx);
    J.warp_begin = warps;
    warps += (unsigned long long)J.n_anchors * (unsigned long long)J.links;
    jobs.push_back(J);
  }
  if (jobs.empty()) return TT_OK;
  if (jobs.size() > e->topn_cap) {
    TT_CK(cudaStreamSynchronize(e->stream));  // the old list may still be read
    dfree(e, e->d_topn);
    e->d_topn = nullptr;
    e->topn_cap = 0;
    TT_CK(dmalloc(e, &e->d_topn, sizeof(TTTopnJob) * jobs.size() * 2));
    e->topn_cap = jobs.size() * 2;
  }
  TT_CK(cudaMemcpyAsync(e->d_topn, jobs.data(), sizeof(TTTopnJob) * jobs.size(), cudaMemcpyHostToDevice, e->stream));
  cudaError_t err = tt_launch_topn_select(e->d_topn, (int)jobs.size(), warps, e->stream);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "tap selection launch: %s", cudaGetErrorString(err));
  ++e->launches;
  return TT_OK;
}

}  // namespace ttx
