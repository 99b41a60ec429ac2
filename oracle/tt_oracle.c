/*
 * tt_oracle.c -- FP64 CPU oracle for the per-UE time-varying multi-tap channel
 * convolution.  TEST INFRASTRUCTURE ONLY: it is called by tests/, by
 * __graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the
 * product path.  It shares no code, header or table with the CUDA library.
 *
 * What it computes, for one UE (each UE is independent: per-UE channel
 * isolation, Sec. III-B and Sec. III-C "Parallelizing Convolution Computation"):
 *
 *   y_r[m] = sum_t sum_k h_{r,t,k}(m) * x_t[m - d_k]  +  w_r[m]          (Sec. III-B, y_u = x * h_u)
 *
 * with
 *   - x_t[m] the complex int16 input of Tx antenna t at absolute sample m,
 *     x_t[m] = 0 before the first processed slot (zero initial delay line);
 *   - h(m) linear between OFDM-symbol anchors:  for b_a <= m < b_a + L_a,
 *       h(m) = H[a] + ((m - b_a) / L_a) * (H[a+1] - H[a]),
 *     where a is the absolute symbol index and b_a its first sample; the
 *     anchor after the last symbol of a slot is the next slot's first symbol;
 *   - H[a] the trace value at anchor a (Sec. IV: discrete complex taps on a
 *     fixed delay grid per time step).  With step_samples == 0 the trace holds
 *     one value per symbol; otherwise trace entry i sits at sample i*step and
 *     H[a] is the linear interpolation in trace time p = b_a / step, in FP64;
 *   - w_r[m] optional AWGN: sigma^2 per complex sample, Gaussian pairs from
 *     Box-Muller on uniforms drawn from Philox4x32-10 (Salmon et al., SC'11)
 *     with key (seed_lo, seed_hi) and counter (p_lo, p_hi, ue_id, r), p = m>>1;
 *     words 0,1 serve even m and words 2,3 odd m;  u = (floor(w/2^9)+0.5)*2^-23;
 *   - q = clamp(round_half_even(y), -32768, 32767), per component.
 *
 * The paper leaves interpolation, anchors, noise and rounding unspecified;
 * these are the readings listed with the design notes.  Everything is FP64
 * and written as plain loops so it can be checked against the formulas by eye.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  Multipliers and Weyl key increments from there. */
/* ------------------------------------------------------------------------- */
#define PHX_M0 0xD2511F53u
#define PHX_M1 0xCD9E8D57u
#define PHX_W0 0x9E3779B9u
#define PHX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHX_M0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)PHX_M1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n1 = lo1;
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  uint32_t n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void tto_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += PHX_W0; k[1] += PHX_W1; }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof c);
}

/* uniform in (0,1) from the top 23 bits of a word */
static double u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* complex AWGN sample for (seed, ue, rx, absolute sample m): out = {re, im} */
void tto_noise(uint64_t seed, uint32_t ue_id, uint32_t rx, uint64_t m, double noise_var,
               double out[2]) {
  uint64_t p = m >> 1;
  uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), ue_id, rx};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  tto_philox4x32_10(ctr, key, w);
  int o = (int)(m & 1u) * 2;
  double u0 = u01(w[o]), u1 = u01(w[o + 1]);
  double r = sqrt(-2.0 * log(u0));
  double th = 2.0 * M_PI * u1;
  double s = sqrt(noise_var / 2.0);
  out[0] = s * r * cos(th);
  out[1] = s * r * sin(th);
}

/* ------------------------------------------------------------------------- */
/* one UE                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint32_t n;               /* samples per slot */
  uint32_t nsym;            /* symbols per slot */
  const uint32_t *sym_len;  /* [nsym], sums to n */
  uint32_t n_tx, n_rx, n_taps;
  const int32_t *delays;    /* [n_taps] */
  const float *taps;        /* complex64 [n_anchors][n_rx][n_tx][n_taps], re/im interleaved */
  uint32_t n_anchors;
  double step_samples;      /* 0: one trace entry per symbol */
  int32_t loop;             /* trace wraps around instead of holding its last entry */
  uint64_t seed;
  uint32_t ue_id;
  double noise_var;         /* sigma^2 per complex sample, 0 = off */
  uint32_t top_n;           /* 0 = every tap; else the top-n taps of each anchor (Sec. III-C) */
  const unsigned char *keep; /* NULL, or an explicit tap selection that replaces the top-n rule:
                                [n_slots*nsym + 1][n_rx][n_tx][n_taps], nonzero = tap used, indexed
                                by the anchor's position in the run (anchor s_first*nsym + i at i) */
} tto_ue;

static uint64_t trace_index(const tto_ue *u, uint64_t i) {
  if (u->loop) return i % u->n_anchors;
  return i < u->n_anchors ? i : (uint64_t)u->n_anchors - 1;
}

static uint64_t symbol_start(const tto_ue *u, uint64_t a) {
  uint64_t s = a / u->nsym, j = a % u->nsym, b = s * u->n;
  for (uint64_t i = 0; i < j; ++i) b += u->sym_len[i];
  return b;
}

/* H[a] for every (r, t, k): out[((r*n_tx + t)*n_taps + k)*2 + {0,1}] */
void tto_anchor(const tto_ue *u, uint64_t a, double *out) {
  size_t per = (size_t)u->n_rx * u->n_tx * u->n_taps;
  if (u->step_samples == 0.0) {
    const float *h = u->taps + 2 * per * trace_index(u, a);
    for (size_t e = 0; e < 2 * per; ++e) out[e] = (double)h[e];
    return;
  }
  double p = (double)symbol_start(u, a) / u->step_samples;
  double i0 = floor(p);
  double f = p - i0;
  const float *h0 = u->taps + 2 * per * trace_index(u, (uint64_t)i0);
  const float *h1 = u->taps + 2 * per * trace_index(u, (uint64_t)i0 + 1);
  for (size_t e = 0; e < 2 * per; ++e)
    out[e] = (double)h0[e] + f * ((double)h1[e] - (double)h0[e]);
}

/* Sparse convolution (Sec. III-C, "top-n dominant taps per time step"):
 * keep[(r*n_tx+t)*n_taps+k] = 1 for the top_n taps of |H[a]|^2 per link, the powers taken in FP64
 * from the FP64 anchor, ties to the lower k.  The selection of anchor a holds for the whole symbol
 * [b_a, b_{a+1}); each kept tap is interpolated toward its own H[a+1]. */
static double tap_power(const double *h) { return h[0] * h[0] + h[1] * h[1]; }

static void top_n_mask(const tto_ue *u, const double *H, unsigned char *keep) {
  for (uint32_t r = 0; r < u->n_rx; ++r)
    for (uint32_t t = 0; t < u->n_tx; ++t) {
      size_t base = ((size_t)r * u->n_tx + t) * u->n_taps;
      for (uint32_t k = 0; k < u->n_taps; ++k) {
        if (u->top_n == 0 || u->top_n >= u->n_taps) { keep[base + k] = 1; continue; }
        /* rank = number of taps that beat tap k */
        const double pk = tap_power(H + 2 * (base + k));
        uint32_t rank = 0;
        for (uint32_t j = 0; j < u->n_taps; ++j) {
          const double pj = tap_power(H + 2 * (base + j));
          if (pj > pk || (pj == pk && j < k)) ++rank;
        }
        keep[base + k] = rank < u->top_n;
      }
    }
}

/*
 * Process slots [s_first, s_first + n_slots) of one UE.
 *   x : int16 [n_tx][n_slots*n][2]   (samples before slot s_first are zero)
 *   y : double [n_rx][n_slots*n][2] or NULL   (before packing)
 *   q : int16  [n_rx][n_slots*n][2] or NULL
 * Returns 0, or -1 on an invalid argument.
 */
int tto_run(const tto_ue *u, uint64_t s_first, uint32_t n_slots, const int16_t *x, double *y,
            int16_t *q, int nthreads) {
  if (!u || !x || u->n == 0 || u->nsym == 0 || u->n_taps == 0 || u->n_anchors == 0) return -1;
  uint64_t tot = 0;
  for (uint32_t j = 0; j < u->nsym; ++j) tot += u->sym_len[j];
  if (tot != u->n) return -1;
  for (uint32_t k = 0; k < u->n_taps; ++k)
    if (u->delays[k] < 0) return -1;

  const size_t per = (size_t)u->n_rx * u->n_tx * u->n_taps;
  const size_t n_anch = (size_t)n_slots * u->nsym + 1;
  double *A = (double *)malloc(sizeof(double) * 2 * per * n_anch);
  unsigned char *keep = (unsigned char *)malloc(per * n_anch);
  uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * u->nsym);
  if (!A || !keep || !start) { free(A); free(keep); free(start); return -1; }
  for (size_t i = 0; i < n_anch; ++i) {
    tto_anchor(u, s_first * u->nsym + i, A + 2 * per * i);
    if (u->keep) memcpy(keep + per * i, u->keep + per * i, per);
    else top_n_mask(u, A + 2 * per * i, keep + per * i);
  }
  start[0] = 0;
  for (uint32_t j = 1; j < u->nsym; ++j) start[j] = start[j - 1] + u->sym_len[j - 1];

  const int64_t total = (int64_t)n_slots * u->n;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t r = 0; r < (int64_t)u->n_rx; ++r) {
    for (int64_t i = 0; i < total; ++i) {
      int64_t sl = i / u->n, w = i % u->n;
      uint32_t j = 0;
      while (j + 1 < u->nsym && (uint32_t)w >= start[j + 1]) ++j;
      double tau = (double)(w - start[j]) / (double)u->sym_len[j];
      size_t a0 = (size_t)sl * u->nsym + j;         /* index into the anchor table */
      const double *H0 = A + 2 * per * a0;
      const double *H1 = A + 2 * per * (a0 + 1);
      const unsigned char *kp = keep + per * a0;
      double acc_re = 0.0, acc_im = 0.0;
      for (uint32_t t = 0; t < u->n_tx; ++t) {
        for (uint32_t k = 0; k < u->n_taps; ++k) {
          size_t e = ((size_t)r * u->n_tx + t) * u->n_taps + k;
          if (!kp[e]) continue;
          double h_re = H0[2 * e] + tau * (H1[2 * e] - H0[2 * e]);
          double h_im = H0[2 * e + 1] + tau * (H1[2 * e + 1] - H0[2 * e + 1]);
          int64_t ii = i - u->delays[k];
          if (ii < 0) continue;
          double x_re = (double)x[((size_t)t * total + ii) * 2];
          double x_im = (double)x[((size_t)t * total + ii) * 2 + 1];
          acc_re += h_re * x_re - h_im * x_im;
          acc_im += h_re * x_im + h_im * x_re;
        }
      }
      if (u->noise_var > 0.0) {
        double nz[2];
        tto_noise(u->seed, u->ue_id, (uint32_t)r, s_first * u->n + (uint64_t)i, u->noise_var, nz);
        acc_re += nz[0];
        acc_im += nz[1];
      }
      size_t o = ((size_t)r * total + i) * 2;
      if (y) { y[o] = acc_re; y[o + 1] = acc_im; }
      if (q) {
        double v[2] = {nearbyint(acc_re), nearbyint(acc_im)};
        for (int c = 0; c < 2; ++c) {
          if (v[c] > 32767.0) v[c] = 32767.0;
          if (v[c] < -32768.0) v[c] = -32768.0;
          q[o + c] = (int16_t)v[c];
        }
      }
    }
  }
  free(A);
  free(keep);
  free(start);
  return 0;
}

/*
 * Uplink aggregation at a cell (Sec. III-A, vanilla rfsim: the gNB convolves each UE's uplink
 * stream with that UE's channel and aggregates the results): for every Rx antenna r and sample i,
 *   y[r][i] = sum over members u (in the given order) of y_u[r][i]  +  w_cell[r][m_first + i]
 * with w_cell the AWGN of the cell's own key (seed, cell_id) at absolute sample m_first + i, then
 * the same round-half-even, saturating packing as tto_run.  The members' y_u come from tto_run with
 * their own noise off.  y (double [n_rx][total][2]) and q (int16 [n_rx][total][2]) may be NULL.
 */
int tto_cell(uint32_t n_members, const double *const *y_members, uint32_t n_rx, uint64_t total,
             uint64_t m_first, uint64_t seed, uint32_t cell_id, double noise_var, double *y, int16_t *q) {
  if (!y_members) return -1;
  for (uint32_t u = 0; u < n_members; ++u)
    if (!y_members[u]) return -1;
  for (uint32_t r = 0; r < n_rx; ++r) {
    for (uint64_t i = 0; i < total; ++i) {
      const size_t o = ((size_t)r * total + i) * 2;
      double acc_re = 0.0, acc_im = 0.0;
      for (uint32_t u = 0; u < n_members; ++u) {
        acc_re += y_members[u][o];
        acc_im += y_members[u][o + 1];
      }
      if (noise_var > 0.0) {
        double nz[2];
        tto_noise(seed, cell_id, r, m_first + i, noise_var, nz);
        acc_re += nz[0];
        acc_im += nz[1];
      }
      if (y) { y[o] = acc_re; y[o + 1] = acc_im; }
      if (q) {
        double v[2] = {nearbyint(acc_re), nearbyint(acc_im)};
        for (int c = 0; c < 2; ++c) {
          if (v[c] > 32767.0) v[c] = 32767.0;
          if (v[c] < -32768.0) v[c] = -32768.0;
          q[o + c] = (int16_t)v[c];
        }
      }
    }
  }
  return 0;
}

int tto_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
