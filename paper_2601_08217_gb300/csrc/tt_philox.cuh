// Counter-based AWGN for the channel kernels.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
// multiplies with the published multipliers, key bumped by the published
// Weyl constants between rounds.  Keying used by the channel path: key =
// (seed_lo, seed_hi), counter = (p_lo, p_hi, ue_id, rx) with p = m >> 1 for
// absolute sample m; words 0,1 feed even m, words 2,3 odd m.  Gaussian pairs
// come from Box-Muller (Box & Muller, 1958) on u = (floor(w / 2^9) + 0.5) 2^-23.
#pragma once
#include <cstdint>

__device__ __forceinline__ uint4 tt_philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// (floor(w / 2^9) + 0.5) * 2^-23, exactly: build 1 + floor(w/2^9) 2^-23 from the bits
// and subtract 1 - 2^-24.  Never 0, never 1.
__device__ __forceinline__ float tt_u01(uint32_t w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994f;
}

// Standard normal pair (r cos th, r sin th) with r = sqrt(-2 ln u0), th = 2 pi u1.
// The angle is evaluated as th - pi = 2 pi u1 - pi, inside the fast sine's
// accurate range, and the signs flipped back.  The radius uses the hardware
// square root (sqrt.approx.f32) of the clamped, non-negative argument.
__device__ __forceinline__ float tt_sqrt_approx(float v) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ float2 tt_box_muller(uint32_t w0, uint32_t w1) {
  const float u0 = tt_u01(w0), u1 = tt_u01(w1);
  const float r = tt_sqrt_approx(fmaxf(-1.38629436111989061f * __log2f(u0), 0.0f));
  float s, c;
  __sincosf(fmaf(6.28318530717958648f, u1, -3.14159265358979324f), &s, &c);
  return make_float2(-r * c, -r * s);
}

// acc += sigma * (Gaussian pair) without forming the pair first.
__device__ __forceinline__ void tt_box_muller_add(uint32_t w0, uint32_t w1, float sigma, float2 &acc) {
  const float u0 = tt_u01(w0), u1 = tt_u01(w1);
  const float r = tt_sqrt_approx(fmaxf(-1.38629436111989061f * __log2f(u0), 0.0f)) * (-sigma);
  float s, c;
  __sincosf(fmaf(6.28318530717958648f, u1, -3.14159265358979324f), &s, &c);
  acc.x = fmaf(r, c, acc.x);
  acc.y = fmaf(r, s, acc.y);
}

// AWGN for samples m and m+1 (m even) of (seed, ue, rx): one Philox block.
__device__ __forceinline__ void tt_awgn_pair(uint64_t seed, uint32_t ue, uint32_t rx, uint64_t m,
                                             float2 &n0, float2 &n1) {
  const uint64_t p = m >> 1;
  const uint4 w = tt_philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), ue, rx),
                                   (uint32_t)seed, (uint32_t)(seed >> 32));
  n0 = tt_box_muller(w.x, w.y);
  n1 = tt_box_muller(w.z, w.w);
}

__device__ __forceinline__ void tt_awgn_add_pair(uint64_t seed, uint32_t ue, uint32_t rx, uint64_t m, float sigma,
                                                 float2 &a0, float2 &a1) {
  const uint64_t p = m >> 1;
  const uint4 w = tt_philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), ue, rx),
                                   (uint32_t)seed, (uint32_t)(seed >> 32));
  tt_box_muller_add(w.x, w.y, sigma, a0);
  tt_box_muller_add(w.z, w.w, sigma, a1);
}

__device__ __forceinline__ void tt_awgn_add_one(uint64_t seed, uint32_t ue, uint32_t rx, uint64_t m, float sigma,
                                                float2 &a) {
  const uint64_t p = m >> 1;
  const uint4 w = tt_philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), ue, rx),
                                   (uint32_t)seed, (uint32_t)(seed >> 32));
  if (m & 1) tt_box_muller_add(w.z, w.w, sigma, a);
  else tt_box_muller_add(w.x, w.y, sigma, a);
}

__device__ __forceinline__ float2 tt_awgn_one(uint64_t seed, uint32_t ue, uint32_t rx, uint64_t m) {
  const uint64_t p = m >> 1;
  const uint4 w = tt_philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), ue, rx),
                                   (uint32_t)seed, (uint32_t)(seed >> 32));
  return (m & 1) ? tt_box_muller(w.z, w.w) : tt_box_muller(w.x, w.y);
}

// clamp(round_half_even(v)) to int16 for I and Q, packed I | Q << 16.
// Adding 1.5 * 2^23 rounds to an integer (round-to-nearest-even) that lands in
// the low mantissa bits; the low 16 bits of each are the two's-complement int16.
__device__ __forceinline__ uint32_t tt_pack_iq(float re, float im) {
  re = fminf(fmaxf(re, -32768.0f), 32767.0f);
  im = fminf(fmaxf(im, -32768.0f), 32767.0f);
  const uint32_t a = __float_as_uint(re + 12582912.0f);
  const uint32_t b = __float_as_uint(im + 12582912.0f);
  return __byte_perm(a, b, 0x5410);
}

__device__ __forceinline__ float2 tt_unpack_iq(uint32_t v) {
  return make_float2((float)(int16_t)(v & 0xFFFFu), (float)(int16_t)(v >> 16));
}
