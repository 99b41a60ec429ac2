// Autotuner of the tiled FP32 kernel and its on-disk cache.
//
// The tiled kernel's geometry per channel is (S samples per thread, TPB threads per CTA); a work
// item, the kernel's tile, spans TPB * S samples of one slot.  The tuner searches both axes for
// every class of channels (same symbol lengths, antennas, tap-count bucket, delay class, AWGN,
// output format, top-n) under one objective: the time of the whole batch as tt_engine_run
// launches it.  Tap counts share a bucket up to the next power of two (at least 8), so channels
// that differ by a few taps tune together and one timing noise cannot split them into more
// kernel variants.
//
// The cache file (named by the environment variable TT_TUNE_CACHE) is plain text, one choice per
// line: device name, SM count, class key, S, TPB, separated by tabs.  An engine reads the lines of
// its own device model when it is created; a channel of a cached class then starts at the cached
// geometry when its trace is loaded.  The tuner writes its choices back, keeping every other line.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <unistd.h>
#include <vector>

#include "tt_chan.h"
#include "tt_engine_impl.h"
#include "tt_internal.h"

using ttx::fail;

namespace {

struct CacheLine {
  std::string device, key;
  int sms = 0, spt = 0, tpb = 0;
};

// Parse one line; false for blank or malformed lines (skipped, never fatal).
bool parse_line(const std::string &line, CacheLine &out) {
  std::vector<std::string> f;
  std::string cur;
  for (char ch : line) {
    if (ch == '\t') {
      f.push_back(cur);
      cur.clear();
    } else if (ch != '\r' && ch != '\n') {
      cur.push_back(ch);
    }
  }
  f.push_back(cur);
  if (f.size() != 5 || f[0].empty() || f[2].empty()) return false;
  char *end = nullptr;
  out.device = f[0];
  out.key = f[2];
  out.sms = (int)std::strtol(f[1].c_str(), &end, 10);
  if (*end || out.sms <= 0) return false;
  out.spt = (int)std::strtol(f[3].c_str(), &end, 10);
  if (*end || out.spt <= 0) return false;
  out.tpb = (int)std::strtol(f[4].c_str(), &end, 10);
  if (*end || out.tpb <= 0) return false;
  return true;
}

std::vector<std::string> read_lines(const std::string &path) {
  std::vector<std::string> out;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) out.push_back(line);
  return out;
}

// Write this engine's choices into the cache file: lines of other device models or classes stay,
// lines of the tuned classes are replaced.  Written to a temporary file, then renamed over.
tt_status tune_save(tt_engine *e) {
  std::lock_guard<std::mutex> lk(e->tune_mu);
  if (e->tune_path.empty()) return TT_OK;
  std::ostringstream out;
  for (const std::string &line : read_lines(e->tune_path)) {
    CacheLine l;
    if (!parse_line(line, l)) continue;
    if (l.device == e->dev_name && l.sms == e->num_sms && e->tune.count(l.key)) continue;
    out << line << "\n";
  }
  for (const auto &kv : e->tune)
    out << e->dev_name << "\t" << e->num_sms << "\t" << kv.first << "\t" << kv.second.first << "\t"
        << kv.second.second << "\n";
  const std::string tmp = e->tune_path + ".tmp" + std::to_string((long long)getpid());
  {
    std::ofstream f(tmp, std::ios::trunc);
    f << out.str();
    f.flush();
    if (!f) {
      std::remove(tmp.c_str());
      return fail(TT_ERR_IO, "tuning cache: cannot write %s", tmp.c_str());
    }
  }
  if (std::rename(tmp.c_str(), e->tune_path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return fail(TT_ERR_IO, "tuning cache: cannot replace %s", e->tune_path.c_str());
  }
  return TT_OK;
}

}  // namespace

namespace ttx {

std::string tune_class_key(const tt_chan *c, uint32_t n_taps, int dclass) {
  std::ostringstream k;
  k << "L=";
  for (size_t j = 0; j < c->sym_len.size(); ++j) k << (j ? "," : "") << c->sym_len[j];
  uint32_t bucket = 8;
  while (bucket < n_taps) bucket *= 2;
  k << ";tx=" << c->cfg.n_tx << ";rx=" << c->cfg.n_rx << ";K<=" << bucket << ";dc=" << dclass
    << ";awgn=" << (c->cfg.noise_var > 0.f ? 1 : 0) << ";cf32=" << (c->cfg.output_format == TT_OUT_CF32 ? 1 : 0)
    << ";top=" << c->cfg.top_n;
  return k.str();
}

uint32_t tune_spt_cap(const tt_engine *e) { return e->spt_override ? e->spt_override : 16; }

bool tune_lookup(tt_engine *e, const std::string &key, int *spt, int *tpb) {
  std::lock_guard<std::mutex> lk(e->tune_mu);
  auto it = e->tune.find(key);
  if (it == e->tune.end()) return false;
  *spt = it->second.first;
  *tpb = it->second.second;
  return true;
}

void tune_load(tt_engine *e) {
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, e->device) == cudaSuccess) e->dev_name = prop.name;
  const char *path = std::getenv("TT_TUNE_CACHE");
  std::lock_guard<std::mutex> lk(e->tune_mu);
  e->tune.clear();
  e->tune_path = path && *path ? path : "";
  if (e->tune_path.empty()) return;
  for (const std::string &line : read_lines(e->tune_path)) {
    CacheLine l;
    if (parse_line(line, l) && l.device == e->dev_name && l.sms == e->num_sms) e->tune[l.key] = {l.spt, l.tpb};
  }
}

}  // namespace ttx

tt_status tt_engine_autotune(tt_engine *e, int32_t reps, uint32_t *classes_tuned) {
  const ttx::NvtxScope nvtx_range("tt autotune");
  if (!e) return fail(TT_ERR_INVALID, "null engine");
  if (reps < 1) reps = 3;
  std::lock_guard<std::mutex> lk(e->mu);
  TT_CK(cudaSetDevice(e->device));
  ttx::sync_all(e);
  std::vector<std::pair<std::string, std::vector<tt_chan *>>> classes;
  for (tt_chan *c : e->table) {
    if (!c || !c->has_trace || c->cfg.precision != TT_FP32) continue;
    const std::string key = ttx::tune_class_key(c, (uint32_t)c->desc.n_taps, c->dclass);
    auto it = std::find_if(classes.begin(), classes.end(), [&](const auto &p) { return p.first == key; });
    if (it == classes.end()) classes.push_back({key, {c}});
    else it->second.push_back(c);
  }
  // The objective is the whole batch: one slot of every channel that has a free ring position,
  // launched as the engine launches it.  A class's geometry is changed only when the batch gets
  // faster, so the tuner never splits the launch into more kernel variants for a class-local gain.
  std::vector<tt_chan *> room;
  std::vector<uint64_t> first, count;
  for (auto &cls : classes)
    for (tt_chan *c : cls.second) {
      const uint64_t f = c->started ? c->pushed_end : 0, start = c->started ? c->pulled_end : 0;
      if (f + 1 - start + (uint64_t)c->hist <= (uint64_t)c->Q) {
        room.push_back(c);
        first.push_back(f);
        count.push_back(1);
      }
    }
  if (room.empty()) {
    if (classes_tuned) *classes_tuned = 0;
    return TT_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  TT_CK(cudaEventCreate(&a));
  TT_CK(cudaEventCreate(&b));
  // largest classes first: their choice moves the batch most
  std::stable_sort(classes.begin(), classes.end(), [](const auto &x, const auto &y) {
    auto work = [](const std::vector<tt_chan *> &v) {
      double w = 0;
      for (const tt_chan *c : v) w += (double)c->n * c->desc.n_taps * c->cfg.n_tx * c->cfg.n_rx;
      return w;
    };
    return work(x.second) > work(y.second);
  });
  float cur_ms = 0.f;
  uint32_t tuned = 0;
  tt_status result = ttx::time_batch(e, room, first, count, reps, a, b, &cur_ms);
  std::vector<std::pair<std::string, std::pair<int, int>>> chosen;
  for (size_t ci = 0; ci < classes.size() && result == TT_OK; ++ci) {
    auto &cls = classes[ci];
    tt_chan *c0 = cls.second[0];
    std::vector<std::pair<int, int>> cands;  // (samples per thread, threads per CTA) that fit every member
    for (int s : ttx::spt_candidates(c0->sym_len, ttx::tune_spt_cap(e), c0->cfg.n_rx, c0->cfg.n_tx))
      for (int t : {TT_TPB, TT_TPB_WIDE}) {
        if (e->tpb_override && t != (int)e->tpb_override) continue;
        bool fit = true;
        for (const tt_chan *c : cls.second) {
          int need = 0;
          fit = fit && ttx::smem_need(c, s, t, &need) != 0;
        }
        if (fit) cands.push_back({s, t});
      }
    const std::pair<int, int> start{c0->spt, c0->tpb};
    std::pair<int, int> best = start;
    if (cands.size() >= 2) {
      for (const auto &g : cands) {
        if (g == start) continue;
        for (tt_chan *c : cls.second)
          if ((result = ttx::apply_geom(c, g.first, g.second)) != TT_OK || (result = ttx::upload_desc(c)) != TT_OK)
            break;
        if (result != TT_OK) break;
        float ms = 0.f, again = 0.f;
        if ((result = ttx::time_batch(e, room, first, count, reps, a, b, &ms)) != TT_OK) break;
        if (ms >= 0.99f * cur_ms) continue;
        // a gain is confirmed by a second timing before it is taken
        if ((result = ttx::time_batch(e, room, first, count, reps, a, b, &again)) != TT_OK) break;
        if (again < 0.99f * cur_ms) {
          cur_ms = std::max(ms, again);
          best = g;
        }
      }
      if (result != TT_OK) break;
      for (tt_chan *c : cls.second)
        if ((result = ttx::apply_geom(c, best.first, best.second)) != TT_OK || (result = ttx::upload_desc(c)) != TT_OK)
          break;
      ++tuned;
    }
    chosen.push_back({cls.first, best});
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ttx::drop_graph(e);  // tuned geometry invalidates the cached graph
  if (result != TT_OK) return result;
  {
    std::lock_guard<std::mutex> tk(e->tune_mu);
    for (const auto &kv : chosen) e->tune[kv.first] = kv.second;
  }
  if ((result = tune_save(e)) != TT_OK) return result;
  if (classes_tuned) *classes_tuned = tuned;
  return TT_OK;
}

tt_status tt_chan_get_geometry(tt_chan *c, tt_chan_geometry *out) {
  if (!c || !c->e || !out) return fail(TT_ERR_INVALID, "null channel or output");
  std::lock_guard<std::mutex> lk(c->e->mu);
  tt_chan_geometry g{};
  g.tensor_core = c->cfg.precision != TT_FP32 ? 1 : 0;
  g.samples_per_thread = g.tensor_core ? 0 : (uint32_t)c->spt;
  g.threads_per_cta = g.tensor_core ? 0 : (uint32_t)c->tpb;
  g.samples_per_item = g.tensor_core ? 0 : (uint32_t)(c->spt * c->tpb);
  g.items_per_slot = (uint32_t)c->desc.items_per_slot;
  g.has_trace = c->has_trace ? 1 : 0;
  *out = g;
  return TT_OK;
}
