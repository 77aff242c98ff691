/*
 * synth.h - seeded synthetic 4+4-bit sample generator (test and benchmark input only).
 *
 * One counter-based definition, implemented twice (CUDA kernel in synth.cu, plain C in
 * synth_host.c), so that device-generated benchmark inputs and host-generated oracle inputs are
 * the same bytes without either side reading the other's output. Holds none of the correlator's
 * arithmetic.
 *
 * Definition
 *   mix(z)      = SplitMix64 finaliser (Steele, Lea & Flood 2014): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
 *                 z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
 *   draw(s, k)  = mix(s + (k + 1) * 0x9E3779B97F4A7C15)            (64-bit wrap-around arithmetic)
 *   Sample (t, c, n) of an array with C channels and N inputs, absolute time t (t0 + local t):
 *   L = (t * C + c) * N + n, h1 = draw(seed, 2L), h2 = draw(seed, 2L + 1).
 *   UNIFORM     byte = h1 & 0xFF  (both nibbles uniform over [-8, 7]).
 *   GAUSS_TONE  per component: noise = sum of the four 16-bit fields of h (h1 for Re, h2 for Im)
 *               minus 131070 (an Irwin-Hall(4) approximation of a Gaussian, std 65536/sqrt(3));
 *               u = unit of the time segment (noise std / u = sigma);
 *               phase p = (t + k[n]) mod 1024; tone_re = tab[p], tone_im = tab[(p + 768) mod 1024]
 *               (tab = round(A u cos(2 pi p / 1024)), computed once on the host and passed in);
 *               q = floor((noise + tone + floor(u / 2)) / u) clipped to [-8, 7].
 *               Segments of seg_len samples alternate unit_lo / unit_hi when sat_period == 2 (odd
 *               segments use unit_hi); the segment with index m8_segment (if >= 0) is all -8-8i.
 */
#ifndef CORR_SYNTH_H
#define CORR_SYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SYNTH_UNIFORM = 0, SYNTH_GAUSS_TONE = 1 };

typedef struct synth_params {
  uint64_t seed;
  int32_t profile;
  int32_t unit_lo;     /* unit for ordinary segments (2200 < unit < 2^25) */
  int32_t unit_hi;     /* unit for odd segments when sat_period == 2 (2200 < unit < 2^25) */
  int32_t sat_period;  /* 0: single unit; 2: alternate segments */
  int32_t seg_len;     /* samples per segment (> 0) */
  int32_t m8_segment;  /* index of the all -8-8i segment, or -1 */
} synth_params;

/* Device: out = uint8[T][C][N] (device pointer), absolute start time t0; tab_lo/tab_hi int32[1024]
 * and k int32[N] are device pointers. Returns 0 or a negative error. Asynchronous on stream. */
int synth_generate_device(uint8_t* out, int T, int C, int N, long long t0, const synth_params* p,
                          const int32_t* tab_lo, const int32_t* tab_hi, const int32_t* k, void* stream);

/* Device, a channel range: out = uint8[T][c_count][N] holding channels c_begin .. c_begin + c_count - 1
 * of an array with C channels (the same bytes as those channels of synth_generate_device's output). */
int synth_generate_device_range(uint8_t* out, int T, int c_begin, int c_count, int C, int N, long long t0,
                                const synth_params* p, const int32_t* tab_lo, const int32_t* tab_hi,
                                const int32_t* k, void* stream);

/* Host: out = uint8[t_count][c_count][N] holding times t0 + t_begin .. and channels c_begin ..
 * of an array with C channels; host pointers. Returns 0 or -1. */
int synth_generate_host(uint8_t* out, int t_begin, int t_count, int c_begin, int c_count, int C, int N,
                        long long t0, const synth_params* p, const int32_t* tab_lo, const int32_t* tab_hi,
                        const int32_t* k);

#ifdef __cplusplus
}
#endif

#endif
