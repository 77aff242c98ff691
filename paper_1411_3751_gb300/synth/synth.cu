// Device implementation of the generator defined in synth.h (one thread per sample).
#include <cuda_runtime.h>
#include "synth.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__device__ __forceinline__ uint64_t draw(uint64_t s, uint64_t k) { return mix64(s + (k + 1ull) * 0x9E3779B97F4A7C15ull); }

// q = floor(x / u) - 64 clipped to [-8, 7], x = noise + tone + 64 u + floor(u / 2). Outside
// [56 u, 72 u) the clip decides; inside, x and u fit 32 bits (u is below 2^25), so the division runs
// in 32-bit unsigned arithmetic and gives the same quotient as the 64-bit definition.
__device__ __forceinline__ int quantise(long long noise, long long tone, long long u) {
  const long long x = noise + tone + 64 * u + u / 2;
  if (x < 56 * u) return -8;
  if (x >= 72 * u) return 7;
  return (int)((unsigned)x / (unsigned)u) - 64;
}

__device__ __forceinline__ long long field_sum(uint64_t h) {
  return (long long)(h & 0xFFFF) + (long long)((h >> 16) & 0xFFFF) + (long long)((h >> 32) & 0xFFFF) +
         (long long)((h >> 48) & 0xFFFF) - 131070;
}

__global__ void synth_kernel(uint8_t* __restrict__ out, long long total, int C, int N, long long t0, synth_params p,
                             const int32_t* __restrict__ tab_lo, const int32_t* __restrict__ tab_hi,
                             const int32_t* __restrict__ k) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(e % N);
    const long long tc = e / N;
    const int c = (int)(tc % C);
    const long long t = t0 + tc / C;
    const uint64_t L = ((uint64_t)t * (uint64_t)C + (uint64_t)c) * (uint64_t)N + (uint64_t)n;
    const uint64_t h1 = draw(p.seed, 2 * L);
    uint8_t b;
    if (p.profile == SYNTH_UNIFORM) {
      b = (uint8_t)(h1 & 0xFF);
    } else {
      const long long seg = t / p.seg_len;
      if (p.m8_segment >= 0 && seg == p.m8_segment) {
        b = 0x88;
      } else {
        const bool hi = (p.sat_period == 2) && (seg % 2 == 1);
        const int32_t* tab = hi ? tab_hi : tab_lo;
        const long long u = hi ? p.unit_hi : p.unit_lo;
        const uint64_t h2 = draw(p.seed, 2 * L + 1);
        const int ph = (int)((t + k[n]) & 1023);
        const int re = quantise(field_sum(h1), tab[ph], u);
        const int im = quantise(field_sum(h2), tab[(ph + 768) & 1023], u);
        b = (uint8_t)(((re & 0xF) << 4) | (im & 0xF));
      }
    }
    out[e] = b;
  }
}

}  // namespace

extern "C" int synth_generate_device(uint8_t* out, int T, int C, int N, long long t0, const synth_params* p,
                                     const int32_t* tab_lo, const int32_t* tab_hi, const int32_t* k, void* stream) {
  if (!out || !p || T < 0 || C < 1 || N < 1) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && (!tab_lo || !k || p->unit_lo <= 2200 || p->unit_lo >= (1 << 25) || p->seg_len <= 0)) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && p->sat_period == 2 && (!tab_hi || p->unit_hi <= 2200 || p->unit_hi >= (1 << 25))) return -1;
  const long long total = (long long)T * C * N;
  if (total == 0) return 0;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  synth_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, total, C, N, t0, *p, tab_lo,
                                                                    tab_hi ? tab_hi : tab_lo, k);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
