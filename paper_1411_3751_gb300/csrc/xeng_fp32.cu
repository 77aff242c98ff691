// FP32 CUDA-core X-engine: the same arithmetic class as the paper's GPU layer (FP32 FMA on CUDA
// cores over 8+8-bit promoted samples, Sec. 2.4-2.5), used as the same-GPU comparison path.
//
// One CTA computes a 64 x 64 block of inputs (i = a-side row block, j = c-side column block,
// block(i) >= block(j), so only the lower block triangle is visited) for one channel. Each of the
// 128 threads holds an 8 (i) x 4 (j) register tile of complex FP32 partial sums. Samples are
// staged per 32-sample slice in shared memory as float2 (sign-extended nibbles). Every
// `flush_len` samples (<= 65536) the partials, which are exact integers of magnitude
// <= 128 * 65536 = 2^23, are converted to int64 and added to the accumulators.
#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int TI = 64, TJ = 64, KT = kF32Kt, NT = 128;
constexpr int UI = 8, UJ = 4;  // per-thread tile

__device__ __forceinline__ float nib(unsigned v) { return (float)(((int)(v & 0xF) ^ 8) - 8); }

__global__ void __launch_bounds__(NT) xeng_fp32_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int npol,
                                                       long long Bs, int flush_len, const int2* __restrict__ tiles,
                                                       long long* __restrict__ cross, long long* __restrict__ autos) {
  __shared__ __align__(16) float2 xi_s[KT][TI];
  __shared__ __align__(16) float2 xj_s[KT][TJ];
  const int2 tb = tiles[blockIdx.x];
  const int f = blockIdx.y;
  const int i0 = tb.x * TI, j0 = tb.y * TJ;
  const int tid = threadIdx.x;
  const int ig = tid >> 4, jg = tid & 15;
  const int P = npol * npol;

  float are[UI][UJ], aim[UI][UJ];
#pragma unroll
  for (int u = 0; u < UI; ++u)
#pragma unroll
    for (int v = 0; v < UJ; ++v) are[u][v] = aim[u][v] = 0.f;

  int since_flush = 0;
  for (int t0 = 0; t0 < T; t0 += KT) {
    __syncthreads();
    for (int e = tid; e < KT * TI; e += NT) {
      const int tt = e / TI, n = e % TI;
      float2 vi = make_float2(0.f, 0.f), vj = make_float2(0.f, 0.f);
      if (t0 + tt < T) {
        const uint8_t* row = in + ((size_t)(t0 + tt) * C + f) * N;
        if (i0 + n < N) {
          const unsigned b = row[i0 + n];
          vi = make_float2(nib(b >> 4), nib(b));
        }
        if (j0 + n < N) {
          const unsigned b = row[j0 + n];
          vj = make_float2(nib(b >> 4), nib(b));
        }
      }
      xi_s[tt][n] = vi;
      xj_s[tt][n] = vj;
    }
    __syncthreads();
#pragma unroll 4
    for (int tt = 0; tt < KT; ++tt) {
      float2 a[UI], b[UJ];
      const float4* pa = reinterpret_cast<const float4*>(&xi_s[tt][ig * UI]);
      const float4* pb = reinterpret_cast<const float4*>(&xj_s[tt][jg * UJ]);
#pragma unroll
      for (int u = 0; u < UI / 2; ++u) {
        const float4 q = pa[u];
        a[2 * u] = make_float2(q.x, q.y);
        a[2 * u + 1] = make_float2(q.z, q.w);
      }
#pragma unroll
      for (int v = 0; v < UJ / 2; ++v) {
        const float4 q = pb[v];
        b[2 * v] = make_float2(q.x, q.y);
        b[2 * v + 1] = make_float2(q.z, q.w);
      }
#pragma unroll
      for (int u = 0; u < UI; ++u)
#pragma unroll
        for (int v = 0; v < UJ; ++v) {
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
      for (int u = 0; u < UI; ++u) {
        const int i = i0 + ig * UI + u;
#pragma unroll
        for (int v = 0; v < UJ; ++v) {
          const int j = j0 + jg * UJ + v;
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
  dim3 grid(n_tiles, s.C);
  xeng_fp32_kernel<<<grid, NT, 0, st>>>(d_in, s.N, s.C, T_blk, s.npol, s.Bs, flush_len, d_tiles, d_cross, d_autos);
  return cudaGetLastError();
}

}  // namespace corr
