/* A plain C user of the channel library: reads one UE's workload from a file, streams its slots
 * through tt_chan_push_slot / tt_engine_run / tt_chan_pull_slot, and writes the int16 output.
 *
 * Input file (little endian):
 *   uint32 N, n_sym, n_taps, n_anchors, n_slots, loop
 *   uint32 symbol_len[n_sym]
 *   int32  delays[n_taps]
 *   float  taps[n_anchors][n_taps][2]      (complex64, one anchor per OFDM symbol, SISO)
 *   int16  iq[n_slots][N][2]
 * Output file: int16 [n_slots][N][2].
 * Exit status: 0 on success, 1 on a file error, 2 on a library error (message on stderr). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "tt_chan.h"

static int lib_fail(const char *what) {
  fprintf(stderr, "%s: %s\n", what, tt_last_error());
  return 2;
}

int main(int argc, char **argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
    return 1;
  }
  FILE *f = fopen(argv[1], "rb");
  if (!f) return 1;
  uint32_t hdr[6];
  if (fread(hdr, sizeof hdr, 1, f) != 1) return 1;
  const uint32_t N = hdr[0], n_sym = hdr[1], K = hdr[2], T = hdr[3], S = hdr[4];
  uint32_t *L = malloc(sizeof(uint32_t) * n_sym);
  int32_t *d = malloc(sizeof(int32_t) * K);
  float *taps = malloc(sizeof(float) * 2 * (size_t)T * K);
  int16_t *iq = malloc(sizeof(int16_t) * 2 * (size_t)S * N);
  int16_t *out = malloc(sizeof(int16_t) * 2 * (size_t)S * N);
  if (!L || !d || !taps || !iq || !out) return 1;
  if (fread(L, sizeof(uint32_t), n_sym, f) != n_sym || fread(d, sizeof(int32_t), K, f) != K ||
      fread(taps, sizeof(float), 2 * (size_t)T * K, f) != 2 * (size_t)T * K ||
      fread(iq, sizeof(int16_t), 2 * (size_t)S * N, f) != 2 * (size_t)S * N)
    return 1;
  fclose(f);
  uint32_t d_max = 0;
  for (uint32_t k = 0; k < K; ++k) d_max = (uint32_t)d[k] > d_max ? (uint32_t)d[k] : d_max;

  tt_engine_config ec = {.struct_size = sizeof(tt_engine_config)}; /* device 0, batched form */
  tt_engine *eng;
  if (tt_engine_create(&ec, &eng) != TT_OK) return lib_fail("tt_engine_create");

  tt_chan_config cc = {.struct_size = sizeof(tt_chan_config)};
  cc.ue_id = 0;
  cc.samples_per_slot = N;
  cc.symbols_per_slot = n_sym;
  cc.symbol_len = L;
  cc.n_tx = 1;
  cc.n_rx = 1;
  cc.max_taps = K;
  cc.max_delay = d_max;
  cc.ring_slots = 0; /* the minimum depth plus two */
  cc.seed = 0;
  cc.noise_var = 0.0f;
  cc.precision = TT_FP32;
  cc.output_format = TT_OUT_INT16;
  tt_chan *ch;
  if (tt_chan_create(eng, &cc, &ch) != TT_OK) return lib_fail("tt_chan_create");

  tt_trace_desc tr = {.struct_size = sizeof(tt_trace_desc)};
  tr.taps = taps;
  tr.delays = d;
  tr.n_anchors = T;
  tr.n_taps = K;
  tr.step_samples = 0.0;
  tr.loop = (int32_t)hdr[5];
  if (tt_chan_load_trace(ch, &tr) != TT_OK) return lib_fail("tt_chan_load_trace");

  /* stream: one slot in, one launch, one slot out */
  for (uint32_t s = 0; s < S; ++s) {
    if (tt_chan_push_slot(ch, s, iq + 2 * (size_t)s * N) != TT_OK) return lib_fail("tt_chan_push_slot");
    if (tt_engine_run(eng) != TT_OK) return lib_fail("tt_engine_run");
    uint64_t got = 0;
    if (tt_chan_pull_slot(ch, &got, out + 2 * (size_t)s * N, -1) != TT_OK) return lib_fail("tt_chan_pull_slot");
    if (got != s) {
      fprintf(stderr, "pulled slot %llu, expected %u\n", (unsigned long long)got, s);
      return 2;
    }
  }
  if (tt_engine_destroy(eng) != TT_OK) return lib_fail("tt_engine_destroy");

  f = fopen(argv[2], "wb");
  if (!f || fwrite(out, sizeof(int16_t), 2 * (size_t)S * N, f) != 2 * (size_t)S * N) return 1;
  fclose(f);
  free(L);
  free(d);
  free(taps);
  free(iq);
  free(out);
  return 0;
}
