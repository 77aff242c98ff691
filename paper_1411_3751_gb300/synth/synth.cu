// Device implementation of the generator defined in synth.h (one thread per 16 consecutive inputs).
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

// One sample: the byte of input n at global index L (t, c fixed by the caller).
__device__ __forceinline__ uint8_t sample_byte(const synth_params& p, uint64_t L, long long t, long long seg, int n,
                                               const int32_t* __restrict__ tab_lo, const int32_t* __restrict__ tab_hi,
                                               const int32_t* __restrict__ k) {
  const uint64_t h1 = draw(p.seed, 2 * L);
  if (p.profile == SYNTH_UNIFORM) return (uint8_t)(h1 & 0xFF);
  if (p.m8_segment >= 0 && seg == p.m8_segment) return 0x88;
  const bool hi = (p.sat_period == 2) && (seg % 2 == 1);
  const int32_t* tab = hi ? tab_hi : tab_lo;
  const long long u = hi ? p.unit_hi : p.unit_lo;
  const uint64_t h2 = draw(p.seed, 2 * L + 1);
  const int ph = (int)((t + k[n]) & 1023);
  const int re = quantise(field_sum(h1), tab[ph], u);
  const int im = quantise(field_sum(h2), tab[(ph + 768) & 1023], u);
  return (uint8_t)(((re & 0xF) << 4) | (im & 0xF));
}

// One thread per 16 consecutive inputs of one (t, c) row: the row arithmetic is done once per 16
// samples and the bytes leave as one 16-byte store where the row allows it.
// Rows cover channels c_begin .. c_begin + c_count - 1 of an array with C channels.
__global__ void synth_kernel(uint8_t* __restrict__ out, long long rows, int c_begin, int c_count, int C, int N,
                             long long t0, synth_params p, const int32_t* __restrict__ tab_lo,
                             const int32_t* __restrict__ tab_hi, const int32_t* __restrict__ k, bool vec) {
  const int chunks = (N + 15) / 16;
  const long long units = rows * chunks;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < units; w += (long long)gridDim.x * blockDim.x) {
    const long long r = w / chunks;
    const int n0 = (int)(w - r * chunks) * 16;
    const long long tl = r / c_count;
    const int c = c_begin + (int)(r - tl * c_count);
    const long long t = t0 + tl;
    const long long seg = p.profile == SYNTH_UNIFORM ? 0 : t / p.seg_len;
    const uint64_t L0 = ((uint64_t)t * (uint64_t)C + (uint64_t)c) * (uint64_t)N + (uint64_t)n0;
    uint8_t* dst = out + r * (long long)N + n0;
    if (vec && n0 + 16 <= N) {
      uint32_t wd[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t v = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = 4 * q + b;
          v |= (uint32_t)sample_byte(p, L0 + j, t, seg, n0 + j, tab_lo, tab_hi, k) << (8 * b);
        }
        wd[q] = v;
      }
      *reinterpret_cast<uint4*>(dst) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    } else {
      for (int j = 0; j < 16 && n0 + j < N; ++j) dst[j] = sample_byte(p, L0 + j, t, seg, n0 + j, tab_lo, tab_hi, k);
    }
  }
}

}  // namespace

extern "C" int synth_generate_device_range(uint8_t* out, int T, int c_begin, int c_count, int C, int N, long long t0,
                                           const synth_params* p, const int32_t* tab_lo, const int32_t* tab_hi,
                                           const int32_t* k, void* stream) {
  if (!out || !p || T < 0 || C < 1 || N < 1 || c_begin < 0 || c_count < 0 || c_begin + c_count > C) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && (!tab_lo || !k || p->unit_lo <= 2200 || p->unit_lo >= (1 << 25) || p->seg_len <= 0)) return -1;
  if (p->profile == SYNTH_GAUSS_TONE && p->sat_period == 2 && (!tab_hi || p->unit_hi <= 2200 || p->unit_hi >= (1 << 25))) return -1;
  const long long rows = (long long)T * c_count;
  if (rows == 0) return 0;
  const long long units = rows * ((N + 15) / 16);
  long long blocks = (units + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  const bool vec = (N % 16) == 0 && (reinterpret_cast<uintptr_t>(out) % 16) == 0;
  synth_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, rows, c_begin, c_count, C, N, t0, *p, tab_lo,
                                                                    tab_hi ? tab_hi : tab_lo, k, vec);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int synth_generate_device(uint8_t* out, int T, int C, int N, long long t0, const synth_params* p,
                                     const int32_t* tab_lo, const int32_t* tab_hi, const int32_t* k, void* stream) {
  return synth_generate_device_range(out, T, 0, C, C, N, t0, p, tab_lo, tab_hi, k, stream);
}
