// FP32 CUDA-core X-engine: the same arithmetic class as the paper's GPU layer (FP32 FMA on CUDA
// cores over 8+8-bit promoted samples, Sec. 2.4-2.5), used as the same-GPU comparison path.
//
// One CTA of 64 threads computes a 64 x 64 block of inputs (i = a-side row block, j = c-side column
// block, block(i) >= block(j), so only the lower block triangle is visited) for one channel. Each
// thread holds an 8 (i) x 8 (j) register tile of complex FP32 partial sums: per sample it reads 8 + 8
// complex values from shared memory and issues 256 FMAs. Samples are staged 32 at a time in shared
// memory as float2 (sign-extended nibbles), in 8-value groups padded against bank conflicts; the raw
// bytes of the next 32 samples are loaded into registers while the current ones are multiplied.
// Every `flush_len` samples (<= 65536) the partials, exact integers of magnitude <= 128 * 65536 = 2^23,
// are converted to int64 and added to the accumulators.
#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int TB = 64, KT = kF32Kt, NT = 64;
constexpr int U = 8;  // per-thread tile: U x U complex
// Shared row of one sample: 8 groups of 8 complex values, each group padded by 2 complex (16 bytes), so
// the 8 column groups a warp reads with 128-bit loads fall into 8 different bank groups.
constexpr int GRP = U + 2, ROW = (TB / U) * GRP;
__device__ __forceinline__ int sx(int n) { return (n / U) * GRP + n % U; }
constexpr int WORDS = KT * 2 * (TB / 4) / NT;  // raw 4-byte words per thread per stage (16)

__device__ __forceinline__ float nib(unsigned v) { return (float)(((int)(v & 0xF) ^ 8) - 8); }

// Raw bytes of inputs x0 + 4 w .. + 3 at time t (zero outside the block or the input range).
__device__ __forceinline__ uint32_t raw_word(const uint8_t* __restrict__ in, int N, int C, int f, int T, int t, int x0,
                                             int w, bool vec) {
  const int n = x0 + 4 * w;
  if (t >= T || n >= N) return 0u;
  const uint8_t* p = in + ((size_t)t * C + f) * N + n;
  if (vec) return __ldg(reinterpret_cast<const unsigned*>(p));  // N % 4 == 0, aligned base
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (n + k < N) v |= (uint32_t)__ldg(p + k) << (8 * k);
  return v;
}

__global__ void __launch_bounds__(NT) xeng_fp32_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int npol,
                                                       long long Bs, int flush_len, const int2* __restrict__ tiles,
                                                       bool vec, long long* __restrict__ cross,
                                                       long long* __restrict__ autos) {
  __shared__ __align__(16) float2 xi_s[KT][ROW];
  __shared__ __align__(16) float2 xj_s[KT][ROW];
  const int2 tb = tiles[blockIdx.x];
  const int f = blockIdx.y;
  const int i0 = tb.x * TB, j0 = tb.y * TB;
  const int tid = threadIdx.x;
  const int ig = tid >> 3, jg = tid & 7;
  const int P = npol * npol;

  // staging: word q of this thread (q < WORDS) = side q / 8, sample (tid + 64 (q % 8)) / 16 ... laid
  // out so that 16 consecutive threads read the 16 words (64 inputs) of one sample row
  uint32_t raw[WORDS];
  auto load = [&](int t0) {
#pragma unroll
    for (int q = 0; q < WORDS; ++q) {
      const int e = tid + NT * (q & 7);  // 0 .. 511 per side
      const int tt = e >> 4, w = e & 15;
      raw[q] = raw_word(in, N, C, f, T, t0 + tt, q < 8 ? i0 : j0, w, vec);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < WORDS; ++q) {
      const int e = tid + NT * (q & 7);
      const int tt = e >> 4, w = e & 15;
      float2* dst = (q < 8 ? &xi_s[tt][sx(4 * w)] : &xj_s[tt][sx(4 * w)]);
      const uint32_t v = raw[q];
      const float4 lo = make_float4(nib(v >> 4), nib(v), nib(v >> 12), nib(v >> 8));
      const float4 hi = make_float4(nib(v >> 20), nib(v >> 16), nib(v >> 28), nib(v >> 24));
      reinterpret_cast<float4*>(dst)[0] = lo;
      reinterpret_cast<float4*>(dst)[1] = hi;
    }
  };

  float are[U][U], aim[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) are[u][v] = aim[u][v] = 0.f;

  int since_flush = 0;
  load(0);
  for (int t0 = 0; t0 < T; t0 += KT) {
    __syncthreads();  // previous stage fully consumed
    store();
    __syncthreads();
    if (t0 + KT < T) load(t0 + KT);  // next stage's bytes in flight during the multiply
#pragma unroll 2
    for (int tt = 0; tt < KT; ++tt) {
      float2 a[U], b[U];
      const float4* pa = reinterpret_cast<const float4*>(&xi_s[tt][ig * GRP]);
      const float4* pb = reinterpret_cast<const float4*>(&xj_s[tt][jg * GRP]);
#pragma unroll
      for (int h = 0; h < U / 2; ++h) {
        const float4 qa = pa[h], qb = pb[h];
        a[2 * h] = make_float2(qa.x, qa.y);
        a[2 * h + 1] = make_float2(qa.z, qa.w);
        b[2 * h] = make_float2(qb.x, qb.y);
        b[2 * h + 1] = make_float2(qb.z, qb.w);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) {
          // x_i conj(x_j) = (ar + i ai)(br - i bi)
          are[u][v] = fmaf(a[u].x, b[v].x, are[u][v]);
          are[u][v] = fmaf(a[u].y, b[v].y, are[u][v]);
          aim[u][v] = fmaf(a[u].y, b[v].x, aim[u][v]);
          aim[u][v] = fmaf(-a[u].x, b[v].y, aim[u][v]);
        }
    }
    since_flush += KT;
    if (since_flush >= flush_len || t0 + KT >= T) {
      since_flush = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + ig * U + u;
#pragma unroll
        for (int v = 0; v < U; ++v) {
          const int j = j0 + jg * U + v;
          const long long re = __float2ll_rn(are[u][v]);
          const long long im = __float2ll_rn(aim[u][v]);
          are[u][v] = aim[u][v] = 0.f;
          if (i >= N || j >= N) continue;
          const int sa = i / npol, sc = j / npol;
          if (sa < sc) continue;
          const long long b = (long long)sa * (sa + 1) / 2 + sc;
          long long* cell = cross + (((long long)f * Bs + b) * P + (i % npol) * npol + (j % npol)) * 2;
          cell[0] += re;
          cell[1] += im;
          if (i == j) autos[(long long)f * N + i] += re;
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_fp32(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const int2* d_tiles,
                        int n_tiles, long long* d_cross, long long* d_autos, cudaStream_t st) {
  if (n_tiles == 0 || T_blk == 0) return cudaSuccess;
  const bool vec = (s.N & 3) == 0 && (reinterpret_cast<uintptr_t>(d_in) & 3) == 0;
  dim3 grid(n_tiles, s.C);
  xeng_fp32_kernel<<<grid, NT, 0, st>>>(d_in, s.N, s.C, T_blk, s.npol, s.Bs, flush_len, d_tiles, vec, d_cross,
                                        d_autos);
  return cudaGetLastError();
}

}  // namespace corr
