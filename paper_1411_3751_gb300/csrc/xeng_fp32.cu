// FP32 CUDA-core X-engine: the same arithmetic class as the paper's GPU layer (FP32 FMA on CUDA
// cores over 8+8-bit promoted samples, Sec. 2.4-2.5), used as the same-GPU comparison path.
//
// One CTA of 64 threads computes a 64 x 64 block of inputs (i = a-side row block, j = c-side column
// block, block(i) >= block(j), so only the lower block triangle is visited) for one channel. Each
// thread holds an 8 (i) x 8 (j) register tile of complex FP32 partial sums as 64 packed pairs: per
// sample it reads 14 128-bit words from shared memory and issues 128 packed f32x2 FMAs (256 FMAs).
// Samples are staged 16 at a time in shared memory (sign-extended nibbles, laid out so that every
// operand pair of a packed FMA is one 64-bit register pair); the raw bytes of the next 16 samples are
// loaded into registers while the current ones are multiplied.
// Every `flush_len` samples (<= 65536) the partials, exact integers of magnitude <= 128 * 65536 = 2^23,
// are converted to int64 and added to the accumulators.
#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int TB = 64, KT = 16, NT = 64;  // KT: samples per shared stage (the path's flush granule is 32)
constexpr int U = 8;                      // per-thread tile: U x U complex
static_assert(kF32Kt % KT == 0, "stages must tile the flush granule");
// Shared rows of one sample, laid out for packed f32x2 FMAs:
//  i side: input n as (re, re, im, im) at AI(n), 8-input groups padded to 36 floats, so the 4 groups a
//          warp reads with 128-bit loads fall into 4 different bank groups;
//  j side: each 8-input group as re[8] | im[8] | -im[8], padded to 28 floats (8 groups per warp, 8
//          different bank groups).
constexpr int GA = 4 * U + 4, ROWA = (TB / U) * GA;
constexpr int GB = 3 * U + 4, ROWB = (TB / U) * GB;
__device__ __forceinline__ int ai_idx(int n) { return (n / U) * GA + (n % U) * 4; }
constexpr int WORDS = KT * 2 * (TB / 4) / NT;  // raw 4-byte words per thread per stage (8)

__device__ __forceinline__ float nib(unsigned v) { return (float)(((int)(v & 0xF) ^ 8) - 8); }

// Packed pair of floats and the packed FMA d = a * b + d on both halves (round to nearest: the
// partial sums here are exact integers below 2^24, so each half equals the scalar FMA chain).
__device__ __forceinline__ unsigned long long pk(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpk(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

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
  __shared__ __align__(16) float xi_s[KT][ROWA];
  __shared__ __align__(16) float xj_s[KT][ROWB];
  const int2 tb = tiles[blockIdx.x];
  const int f = blockIdx.y;
  const int i0 = tb.x * TB, j0 = tb.y * TB;
  const int tid = threadIdx.x;
  const int ig = tid >> 3, jg = tid & 7;
  const int P = npol * npol;

  // staging: word q of this thread (q < WORDS) = side q / 4, sample (tid + 64 (q % 4)) / 16, inputs
  // 4 ((tid + 64 (q % 4)) % 16) ..: 16 consecutive threads read the 16 words (64 inputs) of one sample row
  uint32_t raw[WORDS];
  auto load = [&](int t0) {
#pragma unroll
    for (int q = 0; q < WORDS; ++q) {
      const int e = tid + NT * (q & 3);  // 0 .. 255 per side
      const int tt = e >> 4, w = e & 15;
      raw[q] = raw_word(in, N, C, f, T, t0 + tt, q < 4 ? i0 : j0, w, vec);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < WORDS; ++q) {
      const int e = tid + NT * (q & 3);
      const int tt = e >> 4, w = e & 15;
      const uint32_t v = raw[q];
      float re[4], im[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        re[k] = nib(v >> (8 * k + 4));
        im[k] = nib(v >> (8 * k));
      }
      if (q < 4) {
        float4* dst = reinterpret_cast<float4*>(&xi_s[tt][ai_idx(4 * w)]);
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = make_float4(re[k], re[k], im[k], im[k]);
      } else {
        float* g = &xj_s[tt][(w >> 1) * GB + 4 * (w & 1)];
        *reinterpret_cast<float4*>(g) = make_float4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<float4*>(g + U) = make_float4(im[0], im[1], im[2], im[3]);
        *reinterpret_cast<float4*>(g + 2 * U) = make_float4(-im[0], -im[1], -im[2], -im[3]);
      }
    }
  };

  // accumulator pairs: columns (2 p, 2 p + 1) of row u
  unsigned long long are[U][U / 2], aim[U][U / 2];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int p = 0; p < U / 2; ++p) are[u][p] = aim[u][p] = 0ull;

  int since_flush = 0;
  load(0);
  for (int t0 = 0; t0 < T; t0 += KT) {
    __syncthreads();  // previous stage fully consumed
    store();
    __syncthreads();
    if (t0 + KT < T) load(t0 + KT);  // next stage's bytes in flight during the multiply
#pragma unroll 2
    for (int tt = 0; tt < KT; ++tt) {
      const float4* pa = reinterpret_cast<const float4*>(&xi_s[tt][ig * GA]);
      const float4* pb = reinterpret_cast<const float4*>(&xj_s[tt][jg * GB]);
      unsigned long long ar[U], ai[U], bre[U / 2], bim[U / 2], bnim[U / 2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 q = pa[u];  // (re, re, im, im) of input ig * 8 + u
        ar[u] = pk(q.x, q.y);
        ai[u] = pk(q.z, q.w);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 r = pb[h], m = pb[2 + h], n = pb[4 + h];
        bre[2 * h] = pk(r.x, r.y);
        bre[2 * h + 1] = pk(r.z, r.w);
        bim[2 * h] = pk(m.x, m.y);
        bim[2 * h + 1] = pk(m.z, m.w);
        bnim[2 * h] = pk(n.x, n.y);
        bnim[2 * h + 1] = pk(n.z, n.w);
      }
      // x_i conj(x_j) = (ar + i ai)(br - i bi): re += ar br + ai bi, im += ai br - ar bi, in two sweeps
      // so that the two updates of an accumulator pair are 64 instructions apart (no back-to-back
      // dependence on the FMA latency)
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int p = 0; p < U / 2; ++p) {
          ffma2(are[u][p], ar[u], bre[p]);
          ffma2(aim[u][p], ai[u], bre[p]);
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int p = 0; p < U / 2; ++p) {
          ffma2(are[u][p], ai[u], bim[p]);
          ffma2(aim[u][p], ar[u], bnim[p]);
        }
    }
    since_flush += KT;
    if (since_flush >= flush_len || t0 + KT >= T) {
      since_flush = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + ig * U + u;
#pragma unroll
        for (int p = 0; p < U / 2; ++p) {
          float re2[2], im2[2];
          unpk(are[u][p], re2[0], re2[1]);
          unpk(aim[u][p], im2[0], im2[1]);
          are[u][p] = aim[u][p] = 0ull;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = j0 + jg * U + 2 * p + h;
            const long long re = __float2ll_rn(re2[h]);
            const long long im = __float2ll_rn(im2[h]);
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
