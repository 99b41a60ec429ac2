// Uplink aggregation cells (Sec. III-A: the gNB receives the sum of its UEs' uplink streams): the
// C ABI of cells, and the aggregation step of a run (launch_cells), which sums, in attach order, the
// complex64 outputs of every slot all members have launched, adds the cell's own AWGN and packs.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <utility>
#include <vector>

#include "tt_chan.h"
#include "tt_engine_impl.h"
#include "tt_internal.h"

using ttx::dfree;
using ttx::dmalloc;
using ttx::fail;

namespace ttx {

// Engine lock held: whether launch_cells would aggregate something now (every member started and
// the cell has ring room for slots all members have launched).
bool cells_have_work(const tt_engine *e) {
  for (const tt_cell *cl : e->cells) {
    if (cl->members.empty()) continue;
    uint64_t end = UINT64_MAX;
    bool all_started = true;
    for (const tt_chan *m : cl->members) {
      if (!m->started) { all_started = false; break; }
      end = std::min(end, m->launched_end);
    }
    if (!all_started) continue;
    const uint64_t launched = cl->started ? cl->launched_end : cl->members[0]->start_slot;
    const uint64_t pulled = cl->started ? cl->pulled_end : launched;
    if (std::min<uint64_t>(end, pulled + (uint64_t)cl->Q) > launched) return true;
  }
  return false;
}

tt_status launch_cells(tt_engine *e, std::vector<std::pair<tt_cell *, uint64_t>> &ends) {
  for (tt_cell *cl : e->cells) {
    if (cl->members.empty()) continue;
    bool all_started = true;
    uint64_t end = UINT64_MAX;
    for (tt_chan *m : cl->members) {
      if (!m->started) { all_started = false; break; }
      end = std::min(end, m->launched_end);
    }
    if (!all_started) continue;
    if (!cl->started) {
      const uint64_t s0 = cl->members[0]->start_slot;
      for (tt_chan *m : cl->members)
        if (m->start_slot != s0) return fail(TT_ERR_STATE, "cell %u: members start at different slots", cl->cfg.cell_id);
      cl->started = true;
      cl->launched_end = cl->completed_end = cl->pulled_end = s0;
    }
    end = std::min<uint64_t>(end, cl->pulled_end + (uint64_t)cl->Q);
    if (end <= cl->launched_end) continue;
    if (cl->members.size() > cl->members_cap) return fail(TT_ERR_STATE, "cell %u: member table stale", cl->cfg.cell_id);
    TTCellArgs A{};
    A.ring_out = cl->d_out;
    A.members = cl->d_members;
    A.n_members = (int)cl->members.size();
    A.n = cl->n;
    A.n_rx = (int)cl->cfg.n_rx;
    A.ring_q = cl->Q;
    A.out_f32 = cl->cfg.output_format == TT_OUT_CF32 ? 1 : 0;
    A.cell_id = cl->cfg.cell_id;
    A.seed = cl->cfg.seed;
    A.noise_std = cl->cfg.noise_var > 0.f ? (float)std::sqrt((double)cl->cfg.noise_var / 2.0) : 0.f;
    for (uint64_t s0 = cl->launched_end; s0 < end; s0 += 65535) {
      const uint32_t ns = (uint32_t)std::min<uint64_t>(end - s0, 65535);
      cudaError_t err = tt_launch_cell_reduce(A, s0, ns, e->stream);
      if (err != cudaSuccess) return fail(TT_ERR_CUDA, "cell launch: %s", cudaGetErrorString(err));
      ++e->launches;
    }
    ends.push_back({cl, end});
  }
  return TT_OK;
}

}  // namespace ttx

using ttx::get_event;
using ttx::ring_copy;
using ttx::wait_seq;

tt_status tt_cell_create(tt_engine *e, const tt_cell_config *cfg, tt_cell **out) {
  if (!e || !cfg || !out || cfg->struct_size < sizeof(tt_cell_config)) return fail(TT_ERR_INVALID, "tt_cell_create: bad config");
  if (cfg->samples_per_slot == 0 || cfg->samples_per_slot > (1u << 24) || (cfg->samples_per_slot & 1))
    return fail(TT_ERR_INVALID, "cell samples_per_slot must be even, 2 .. 2^24");
  if (cfg->n_rx < 1 || cfg->n_rx > TT_MAX_ANT) return fail(TT_ERR_INVALID, "cell n_rx must be 1..%d", TT_MAX_ANT);
  if (cfg->output_format > TT_OUT_CF32) return fail(TT_ERR_INVALID, "unknown output_format");
  if (!(cfg->noise_var >= 0.0f) || !std::isfinite(cfg->noise_var)) return fail(TT_ERR_INVALID, "bad noise_var");
  const int Q = cfg->ring_slots ? (int)cfg->ring_slots : 4;
  if (Q < 1 || Q > (1 << 20)) return fail(TT_ERR_INVALID, "cell ring_slots out of range");
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  // With a cell, every later batch launches on the engine stream; batches launched so far may
  // still run on other launch lanes, so that stream first waits for all of them.
  for (const auto &p : e->events) TT_CK(cudaStreamWaitEvent(e->stream, p.second, 0));
  const size_t out_e = (size_t)cfg->n_rx * cfg->samples_per_slot * (cfg->output_format == TT_OUT_CF32 ? 4 : 2);
  const uint64_t bytes = (uint64_t)Q * out_e * sizeof(int16_t);
  if (e->budget && e->in_use + bytes > e->budget)
    return fail(TT_ERR_NO_MEMORY, "admission refused: %llu B needed", (unsigned long long)bytes);
  tt_cell *cl = new tt_cell();
  cl->e = e;
  cl->cfg = *cfg;
  cl->n = (int)cfg->samples_per_slot;
  cl->Q = Q;
  cl->slot_out_elems = out_e;
  cudaError_t err = dmalloc(e, &cl->d_out, (size_t)Q * out_e * sizeof(int16_t));
  if (err == cudaSuccess) err = cudaMemsetAsync(cl->d_out, 0, (size_t)Q * out_e * sizeof(int16_t), e->stream);
  if (err != cudaSuccess) {
    dfree(e, cl->d_out);
    delete cl;
    return fail(err == cudaErrorMemoryAllocation ? TT_ERR_NO_MEMORY : TT_ERR_CUDA, "cell ring: %s", cudaGetErrorString(err));
  }
  cl->ring_bytes = bytes;
  e->in_use += bytes;
  e->cells.push_back(cl);
  *out = cl;
  return TT_OK;
}

tt_status tt_cell_attach(tt_cell *cl, tt_chan *c) {
  if (!cl || !cl->e || !c || c->e != cl->e) return fail(TT_ERR_INVALID, "tt_cell_attach: bad cell or channel");
  tt_engine *e = cl->e;
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  if (c->cell) return fail(TT_ERR_STATE, "channel already attached to a cell");
  if (c->started || cl->started) return fail(TT_ERR_STATE, "attach before the first push");
  if (c->n != cl->n || c->cfg.n_rx != cl->cfg.n_rx)
    return fail(TT_ERR_INVALID, "member must have the cell's samples_per_slot and n_rx");
  if (c->cfg.output_format != TT_OUT_CF32 || c->cfg.noise_var != 0.f)
    return fail(TT_ERR_INVALID, "member must have TT_OUT_CF32 output and noise_var 0");
  if (cl->members.size() + 1 > cl->members_cap) {
    const size_t cap = std::max<size_t>(8, 2 * cl->members_cap);
    TTCellMember *d = nullptr;
    TT_CK(cudaStreamSynchronize(e->stream));  // the old table may still be read
    TT_CK(dmalloc(e, &d, sizeof(TTCellMember) * cap));
    dfree(e, cl->d_members);
    cl->d_members = d;
    cl->members_cap = cap;
  }
  cl->members.push_back(c);
  c->cell = cl;
  std::vector<TTCellMember> h(cl->members.size());
  for (size_t i = 0; i < h.size(); ++i) {
    h[i].ring_out = reinterpret_cast<const float2 *>(cl->members[i]->d_out);
    h[i].ring_q = cl->members[i]->Q;
  }
  TT_CK(cudaMemcpy(cl->d_members, h.data(), sizeof(TTCellMember) * h.size(), cudaMemcpyHostToDevice));
  // copies from pageable memory may return before the DMA lands, and the engine's non-blocking
  // streams are not ordered after the default stream: let them land before any kernel reads them
  TT_CK(cudaStreamSynchronize(nullptr));
  return TT_OK;
}

tt_status tt_cell_pull_slots(tt_cell *cl, uint64_t first, uint32_t n, void *out, int64_t timeout_us) {
  const ttx::NvtxScope nvtx_range("tt cell pull");
  if (!cl || !cl->e || (!out && n)) return fail(TT_ERR_INVALID, "tt_cell_pull_slots: bad argument");
  if (n == 0) return TT_OK;
  tt_engine *e = cl->e;
  std::unique_lock<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  if (!cl->started || first != cl->pulled_end)
    return fail(TT_ERR_STATE, "cell pull must start at the oldest unpulled slot %llu", (unsigned long long)cl->pulled_end);
  if (first + n > cl->launched_end) return fail(TT_ERR_AGAIN, "cell slot not aggregated yet");
  uint64_t need = 0;
  for (auto &p : cl->inflight)
    if (p.first >= first + n) { need = p.second; break; }
  if (need && need > e->completed_seq) {
    tt_status s = wait_seq(e, need, timeout_us, lk);
    if (s != TT_OK) return s;
  }
  while (!cl->inflight.empty() && cl->inflight.front().second <= e->completed_seq) cl->inflight.pop_front();
  cudaEvent_t ev = get_event(e);
  if (!ev) return fail(TT_ERR_CUDA, "event creation failed");
  cudaError_t err = ring_copy(cl->d_out, cl->slot_out_elems, cl->Q, first, n, nullptr, out, cudaMemcpyDeviceToHost,
                              e->copy, false);
  if (err == cudaSuccess) err = cudaEventRecord(ev, e->copy);
  if (err == cudaSuccess) {
    lk.unlock();
    err = cudaEventSynchronize(ev);
    lk.lock();
  }
  e->pool.push_back(ev);
  if (err != cudaSuccess) return fail(TT_ERR_CUDA, "cell pull copy: %s", cudaGetErrorString(err));
  cl->pulled_end = first + n;
  return TT_OK;
}

tt_status tt_cell_destroy(tt_cell *cl) {
  if (!cl || !cl->e) return fail(TT_ERR_INVALID, "null cell");
  tt_engine *e = cl->e;
  std::lock_guard<std::mutex> lk(e->mu);
  cudaSetDevice(e->device);
  ttx::sync_all(e);
  for (tt_chan *m : cl->members) m->cell = nullptr;
  dfree(e, cl->d_out);
  dfree(e, cl->d_members);
  e->in_use -= cl->ring_bytes;
  e->cells.erase(std::remove(e->cells.begin(), e->cells.end(), cl), e->cells.end());
  cl->e = nullptr;
  delete cl;
  return TT_OK;
}
