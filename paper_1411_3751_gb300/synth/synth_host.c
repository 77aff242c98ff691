/* Host implementation of the generator defined in synth.h. */
#include <stddef.h>

#include "synth.h"

static uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

static uint64_t draw(uint64_t s, uint64_t k) { return mix64(s + (k + 1ull) * 0x9E3779B97F4A7C15ull); }

static int quantise(int64_t noise, int64_t tone, int64_t u) {
  int64_t x = noise + tone + 64 * u + u / 2; /* > 0 for the admitted units */
  int64_t q = x / u - 64;
  if (q < -8) q = -8;
  if (q > 7) q = 7;
  return (int)q;
}

static int64_t field_sum(uint64_t h) {
  return (int64_t)(h & 0xFFFF) + (int64_t)((h >> 16) & 0xFFFF) + (int64_t)((h >> 32) & 0xFFFF) +
         (int64_t)((h >> 48) & 0xFFFF) - 131070;
}

int synth_generate_host(uint8_t* out, int t_begin, int t_count, int c_begin, int c_count, int C, int N,
                        long long t0, const synth_params* p, const int32_t* tab_lo, const int32_t* tab_hi,
                        const int32_t* k) {
  if (!out || !p || C < 1 || N < 1 || t_count < 0 || c_count < 0 || c_begin < 0 || c_begin + c_count > C) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && (!tab_lo || !k || p->unit_lo <= 2200 || p->unit_lo >= (1 << 25) || p->seg_len <= 0)) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && p->sat_period == 2 && (!tab_hi || p->unit_hi <= 2200 || p->unit_hi >= (1 << 25))) return -1;
  for (int tt = 0; tt < t_count; ++tt) {
    const long long t = t0 + t_begin + tt;
    for (int cc = 0; cc < c_count; ++cc) {
      const int c = c_begin + cc;
      uint8_t* row = out + ((size_t)tt * c_count + cc) * N;
      for (int n = 0; n < N; ++n) {
        const uint64_t L = ((uint64_t)t * (uint64_t)C + (uint64_t)c) * (uint64_t)N + (uint64_t)n;
        const uint64_t h1 = draw(p->seed, 2 * L);
        if (p->profile == SYNTH_UNIFORM) {
          row[n] = (uint8_t)(h1 & 0xFF);
          continue;
        }
        const long long seg = t / p->seg_len;
        if (p->m8_segment >= 0 && seg == p->m8_segment) {
          row[n] = 0x88;
          continue;
        }
        const int hi = (p->sat_period == 2) && (seg % 2 == 1);
        const int32_t* tab = hi ? tab_hi : tab_lo;
        const int64_t u = hi ? p->unit_hi : p->unit_lo;
        const uint64_t h2 = draw(p->seed, 2 * L + 1);
        const int ph = (int)((t + k[n]) & 1023);
        const int re = quantise(field_sum(h1), tab[ph], u);
        const int im = quantise(field_sum(h2), tab[(ph + 768) & 1023], u);
        row[n] = (uint8_t)(((re & 0xF) << 4) | (im & 0xF));
      }
    }
  }
  return 0;
}
