// tt_conv_static: the channel convolution for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to call cudaMalloc at all. Examples: code that
// runs inside another framework's memory pool or a pre-sized real-time
// partition, or a caller that has to keep a fixed memory footprint. The engine
// path (tt_engine_*/tt_chan_*) allocates rings, traces and work lists, so such
// callers cannot use it. This entry point runs the same tiled kernel on
// buffers the caller already owns. The only scratch it needs (UE descriptors,
// the work list, chunk tables, delays, work counters) lives in one file-scope
// __device__ array of fixed size. Every GPU that loads this library holds that
// array until the process exits.
//
// Setup: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress, with that device current, and remembers it. Host code
// must never pass the array's name to a kernel: in host code the name is a
// host-side stand-in, not the device address.
//
// Sharing: all calls use the same array, and it keeps the last call's
// contents. Each call rewrites everything it reads and zeroes its work
// counters. Calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array. Order them on one stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "tt_chan.h"
#include "tt_internal.h"

namespace {

constexpr int kMaxChans = TT_STATIC_MAX_CHANS;
constexpr int kMaxItems = TT_STATIC_MAX_ITEMS_PER_SLOT;
constexpr int kMaxTaps = TT_MAX_TAPS;

// Fixed layout of the scratch array (byte offsets, each 256-aligned).
constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffDesc = 0;
constexpr size_t kOffSeg = align256(kOffDesc + sizeof(TTUEDesc) * kMaxChans);
constexpr size_t kOffChunk = align256(kOffSeg + sizeof(TTSeg) * kMaxChans);
constexpr size_t kOffDelay = align256(kOffChunk + sizeof(int32_t) * kMaxItems * kMaxChans);
constexpr size_t kOffCount = align256(kOffDelay + sizeof(int32_t) * kMaxTaps * kMaxChans);
constexpr size_t kScratchBytes = align256(kOffCount + sizeof(uint32_t) * kMaxChans);

__device__ __align__(256) unsigned char tt_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch[kMaxDevices] = {};

int32_t err(int32_t status, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return tt_set_error(status, buf);
}

}  // namespace

extern "C" tt_status tt_conv_static(const tt_static_chan *chans, uint32_t n_chans, void *stream) {
  if (!chans && n_chans) return err(TT_ERR_INVALID, "tt_conv_static: null chans");
  if (n_chans == 0) return TT_OK;
  if (n_chans > (uint32_t)kMaxChans)
    return err(TT_ERR_INVALID, "tt_conv_static: %u channels, at most %d per call", n_chans, kMaxChans);

  // ---- validate and describe every channel (host only) ----
  std::vector<TTUEDesc> desc(n_chans);
  std::vector<int32_t> chunk_host((size_t)kMaxItems * n_chans, 0), delay_host((size_t)kMaxTaps * n_chans, 0);
  struct Meta { int spt, dclass, tap_need, ntx, nrx, K; uint32_t n_slots; uint64_t first; };
  std::vector<Meta> meta(n_chans);
  for (uint32_t i = 0; i < n_chans; ++i) {
    const tt_static_chan &c = chans[i];
    if (c.struct_size < sizeof(tt_static_chan)) return err(TT_ERR_INVALID, "chan %u: bad struct_size", i);
    const uint32_t N = c.samples_per_slot;
    if (N == 0 || N > (uint32_t)(kMaxItems * TT_TPB))
      return err(TT_ERR_INVALID, "chan %u: samples_per_slot must be 1..%d here", i, kMaxItems * TT_TPB);
    if (c.symbols_per_slot == 0 || c.symbols_per_slot > TT_MAX_SYM || !c.symbol_len)
      return err(TT_ERR_INVALID, "chan %u: symbols_per_slot must be 1..%d", i, TT_MAX_SYM);
    if (c.n_tx < 1 || c.n_tx > TT_MAX_ANT || c.n_rx < 1 || c.n_rx > TT_MAX_ANT)
      return err(TT_ERR_INVALID, "chan %u: n_tx and n_rx must be 1..%d", i, TT_MAX_ANT);
    if (c.n_taps < 1 || c.n_taps > (uint32_t)kMaxTaps || !c.delays || !c.d_taps || c.n_anchors == 0)
      return err(TT_ERR_INVALID, "chan %u: need 1..%d taps, host delays, device taps, >= 1 anchor", i, kMaxTaps);
    if (!c.d_ring_in || !c.d_ring_out) return err(TT_ERR_INVALID, "chan %u: null ring", i);
    if (c.output_format > TT_OUT_CF32) return err(TT_ERR_INVALID, "chan %u: unknown output_format", i);
    // the kernel stages the input ring with 16-byte copies, reads taps as 8-byte complex64 and stores
    // 4-byte packed IQ or 8-byte complex64 outputs
    const uintptr_t out_align = c.output_format == TT_OUT_CF32 ? 8 : 4;
    if ((reinterpret_cast<uintptr_t>(c.d_ring_in) & 15) || (reinterpret_cast<uintptr_t>(c.d_taps) & 7) ||
        (reinterpret_cast<uintptr_t>(c.d_ring_out) & (out_align - 1)))
      return err(TT_ERR_INVALID,
                 "chan %u: d_ring_in must be 16-byte aligned, d_taps 8-byte, d_ring_out %u-byte", i,
                 (unsigned)out_align);
    if (!(c.step_samples >= 0.0) || !std::isfinite(c.step_samples) || !(c.noise_var >= 0.f) ||
        !std::isfinite(c.noise_var))
      return err(TT_ERR_INVALID, "chan %u: bad step_samples or noise_var", i);
    std::vector<uint32_t> L(c.symbol_len, c.symbol_len + c.symbols_per_slot);
    uint64_t sum = 0;
    for (uint32_t v : L) sum += v;
    if (sum != N) return err(TT_ERR_INVALID, "chan %u: symbol lengths do not sum to samples_per_slot", i);
    int d_max = 0;
    for (uint32_t k = 0; k < c.n_taps; ++k) {
      const int32_t d = c.delays[k];
      if (d < 0 || d > TT_MAX_DELAY || (k && d < c.delays[k - 1]))
        return err(TT_ERR_INVALID, "chan %u: delays must be non-decreasing in 0..%d", i, TT_MAX_DELAY);
      d_max = std::max(d_max, (int)d);
    }
    // slot s reads its delay line from the positions of slots s - hist .. s - 1; those of slots before
    // first_slot must not be positions that this call's own slots occupy
    const uint64_t hist = ((uint64_t)d_max + N - 1) / N;
    if ((uint64_t)c.ring_slots < (uint64_t)c.n_slots + hist || c.ring_slots == 0)
      return err(TT_ERR_INVALID, "chan %u: ring_slots %u < n_slots %u + %llu history slot(s) of the delay line", i,
                 c.ring_slots, c.n_slots, (unsigned long long)hist);
    const int dclass = d_max <= TT_DCLASS0 ? 0 : d_max <= TT_DCLASS1 ? 1 : d_max <= TT_DCLASS2 ? 2 : 3;
    // largest samples-per-thread (<= 8) dividing every symbol length and fitting shared memory
    int spt = 0, tap_need = 0, items = 0;
    std::vector<int32_t> L32(L.begin(), L.end()), chunks(kMaxItems);
    for (int s : {8, 4, 2, 1}) {
      bool ok = true;
      for (uint32_t v : L) ok = ok && (v % (uint32_t)s == 0);
      if (!ok) continue;
      const int it = tt_conv_chunk_info(s, TT_TPB, L32.data(), (int)L32.size(), chunks.data(), kMaxItems);
      if (it < 0) continue;
      int touched = 1;
      for (int q = 0; q < it; ++q) touched = std::max(touched, (int)(chunks[q] >> 16));
      const int need = touched * (int)(c.n_rx * c.n_tx * c.n_taps);
      if (tt_conv_smem_bytes(s, TT_TPB, dclass, (int)c.n_tx, need, (int)c.n_taps) <= 200 * 1024) {
        spt = s;
        tap_need = need;
        items = it;
        break;
      }
    }
    if (spt == 0) return err(TT_ERR_INVALID, "chan %u: too large for the tiled kernel", i);
    std::copy(chunks.begin(), chunks.begin() + items, chunk_host.begin() + (size_t)i * kMaxItems);
    std::copy(c.delays, c.delays + c.n_taps, delay_host.begin() + (size_t)i * kMaxTaps);

    TTUEDesc &d = desc[i];
    std::memset(&d, 0, sizeof d);
    d.ring_in = c.d_ring_in;
    d.ring_out = c.d_ring_out;
    d.taps = reinterpret_cast<const float2 *>(c.d_taps);
    d.step_samples = c.step_samples;
    d.seed = c.seed;
    d.n = (int)N;
    d.nsym = (int)c.symbols_per_slot;
    d.n_tx = (int)c.n_tx;
    d.n_rx = (int)c.n_rx;
    d.n_taps = (int)c.n_taps;
    d.d_max = d_max;
    d.ring_q = (int)c.ring_slots;
    d.n_anchors = (int)c.n_anchors;
    d.loop = c.loop ? 1 : 0;
    d.ue_id = c.ue_id;
    d.noise_std = c.noise_var > 0.f ? (float)std::sqrt((double)c.noise_var / 2.0) : 0.f;
    d.out_f32 = c.output_format == TT_OUT_CF32 ? 1 : 0;
    d.top_n = 0;
    d.spt = spt;
    d.tpb = TT_TPB;
    d.dpad = (d_max + spt - 1) / spt * spt;
    d.groups = (int)N / spt;
    d.items_per_slot = items;
    int b = 0, g = 0;
    for (int j = 0; j < d.nsym; ++j) {
      d.sym_start[j] = b;
      d.grp_start[j] = g;
      b += (int)L[j];
      g += (int)L[j] / spt;
    }
    d.sym_start[d.nsym] = b;
    d.grp_start[d.nsym] = g;
    meta[i] = {spt, dclass, tap_need, (int)c.n_tx, (int)c.n_rx, (int)c.n_taps, c.n_slots, c.first_slot};
  }

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return err(TT_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));
  if (dev < 0 || dev >= kMaxDevices) return err(TT_ERR_INVALID, "device %d out of range", dev);
  unsigned char *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch[dev]) {
      void *p = nullptr;
      ce = cudaGetSymbolAddress(&p, tt_static_scratch);
      if (ce != cudaSuccess || !p) return err(TT_ERR_CUDA, "scratch lookup: %s", cudaGetErrorString(ce));
      g_scratch[dev] = static_cast<unsigned char *>(p);
    }
    scratch = g_scratch[dev];
  }
  for (uint32_t i = 0; i < n_chans; ++i) {  // descriptor pointers into the scratch array
    desc[i].delays = reinterpret_cast<int32_t *>(scratch + kOffDelay) + (size_t)i * kMaxTaps;
    desc[i].chunk_info = reinterpret_cast<int32_t *>(scratch + kOffChunk) + (size_t)i * kMaxItems;
  }
  TTUEDesc *d_desc = reinterpret_cast<TTUEDesc *>(scratch + kOffDesc);
  TTSeg *d_seg = reinterpret_cast<TTSeg *>(scratch + kOffSeg);
  int32_t *d_chunk = reinterpret_cast<int32_t *>(scratch + kOffChunk);
  int32_t *d_delay = reinterpret_cast<int32_t *>(scratch + kOffDelay);
  uint32_t *d_count = reinterpret_cast<uint32_t *>(scratch + kOffCount);

  // ---- work list: one run of slots per channel, grouped by kernel variant ----
  std::vector<uint32_t> order(n_chans);
  for (uint32_t i = 0; i < n_chans; ++i) order[i] = i;
  auto key = [&](uint32_t i) {
    return ((meta[i].spt * 8 + meta[i].nrx) * 8 + meta[i].ntx) * 8 + meta[i].dclass;
  };
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key(a) < key(b); });
  std::vector<TTSeg> segs;
  struct Group { int key; size_t seg0; int nseg; uint32_t items; int spt, nrx, ntx, dclass, tap_max, k_max; };
  std::vector<Group> groups;
  for (uint32_t oi = 0; oi < n_chans; ++oi) {
    const uint32_t i = order[oi];
    if (meta[i].n_slots == 0) continue;
    if (groups.empty() || groups.back().key != key(i))
      groups.push_back({key(i), segs.size(), 0, 0, meta[i].spt, meta[i].nrx, meta[i].ntx, meta[i].dclass, 1, 1});
    Group &gr = groups.back();
    TTSeg s{};
    s.first_slot = meta[i].first;
    s.ue = i;
    s.n_slots = meta[i].n_slots;
    s.item_begin = gr.items;
    s.items = meta[i].n_slots * (uint32_t)desc[i].items_per_slot;
    gr.items += s.items;
    gr.tap_max = std::max(gr.tap_max, meta[i].tap_need);
    gr.k_max = std::max(gr.k_max, meta[i].K);
    ++gr.nseg;
    segs.push_back(s);
  }
  if (groups.empty()) return TT_OK;

  // ---- upload into the scratch array (stream-ordered; no allocation) and launch ----
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ce = cudaMemcpyAsync(d_desc, desc.data(), sizeof(TTUEDesc) * n_chans, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d_seg, segs.data(), sizeof(TTSeg) * segs.size(), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d_chunk, chunk_host.data(), sizeof(int32_t) * chunk_host.size(), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d_delay, delay_host.data(), sizeof(int32_t) * delay_host.size(), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d_count, 0, sizeof(uint32_t) * groups.size(), st);
  if (ce != cudaSuccess) return err(TT_ERR_CUDA, "scratch upload: %s", cudaGetErrorString(ce));
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const Group &gr = groups[gi];
    TTLaunch L{};
    L.ues = d_desc;
    L.segs = d_seg + gr.seg0;
    L.n_segs = gr.nseg;
    L.total_items = gr.items;
    L.counter = d_count + gi;
    L.spt = gr.spt;
    L.tpb = TT_TPB;
    L.nrx = gr.nrx;
    L.ntx = gr.ntx;
    L.dclass = gr.dclass;
    L.tap_max = gr.tap_max;
    L.k_max = gr.k_max;
    L.smem = tt_conv_smem_bytes(gr.spt, TT_TPB, gr.dclass, gr.ntx, gr.tap_max, gr.k_max);
    L.grid = -1;
    ce = tt_launch_conv_fp32(L, st);
    if (ce != cudaSuccess) return err(TT_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(ce));
    L.grid = (int)std::min<uint64_t>((uint64_t)(-L.grid) * (uint64_t)sms, gr.items);
    ce = tt_launch_conv_fp32(L, st);
    if (ce != cudaSuccess) return err(TT_ERR_CUDA, "launch: %s", cudaGetErrorString(ce));
  }
  return TT_OK;
}
