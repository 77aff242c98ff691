// Requantiser and corner turn: the tail of the F-engine (Sec. 2.2, FPGA layer). The PFB output of
// each input, 18+18-bit integers (int32 pairs) or float32 complex, is scaled by a digital gain (one
// factor across the band, or one per channel), rounded to the nearest integer (ties to even),
// clipped to 4 bits per component, packed Re << 4 | Im, and written channel-selected and
// corner-turned ([N][T][F] -> [T][C][N]) as the X-engine input.
//
// Per component: x = fl32(gain * v) (one IEEE single-precision product, v converted to float
// first), q = clip(round-half-even(x), lo, 7) with lo = -8 (or -7 when symmetric), NaN -> 0.
//
// HBM-bound transpose: a block stages a 128-channel x 32-input tile of one time sample in shared
// memory. Each warp reads 128 consecutive channels of 4 inputs (1 KiB contiguous per input row) and
// the block writes 128 output rows of 32 consecutive input bytes.
#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int RQ_CH = 128, RQ_IN = 32, RQ_NT = 256;
constexpr int RQ_CPL = RQ_CH / 32;            // channels per lane (4)
constexpr int RQ_IPW = RQ_IN / (RQ_NT / 32);  // inputs per warp (4)

// x = fl32(g v); round to nearest even with cvt.rni (NaN converts to 0, out-of-range values saturate),
// then clip to [lo, 7].
__device__ __forceinline__ unsigned quant4(float v, float g, int lo) {
  const int q = __float2int_rn(__fmul_rn(g, v));
  return (unsigned)min(max(q, lo), 7) & 0xFu;
}

template <typename T2>
__device__ __forceinline__ float2 as_float2(const T2& v);
template <>
__device__ __forceinline__ float2 as_float2<int2>(const int2& v) {
  return make_float2(__int2float_rn(v.x), __int2float_rn(v.y));
}
template <>
__device__ __forceinline__ float2 as_float2<float2>(const float2& v) {
  return v;
}

// Position of a block in its sequence of steps: item = (input tile nt, time t), chunk of channels.
// Items advance by gridDim.x = (dnt, dt) in (tile, time) coordinates; no division per step.
struct RqIter {
  int nt, t, chunk;
  __device__ __forceinline__ void next(int chunks, int tiles_n, int dnt, int dt) {
    if (++chunk == chunks) {
      chunk = 0;
      nt += dnt;
      t += dt;
      if (nt >= tiles_n) {
        nt -= tiles_n;
        ++t;
      }
    }
  }
};

// Persistent: work item w = (input tile w % tiles_n, time sample w / tiles_n); block b takes items
// b, b + gridDim.x, ... and walks each item's rows across the selected channels in 128-channel
// chunks. Blocks running together hold consecutive time samples of every input tile. Warp w owns
// inputs n0 + 4 w .. + 3 and lane l channels c0 + l + 32 k, so a thread packs its four inputs' bytes
// into one 32-bit shared-memory store per channel; the next chunk's 16 loads are in flight while the
// current tile is written out.
template <typename T2>
__global__ void __launch_bounds__(RQ_NT) requant_kernel(const T2* __restrict__ in, int N, int T, int F, int chan0,
                                                        int C, float gain, const float* __restrict__ gains, int lo,
                                                        bool words, uint8_t* __restrict__ out) {
  __shared__ __align__(16) uint8_t tile[RQ_CH][RQ_IN + 4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_n = (N + RQ_IN - 1) / RQ_IN, chunks = (C + RQ_CH - 1) / RQ_CH;
  const int dnt = (int)(gridDim.x % (unsigned)tiles_n), dt = (int)(gridDim.x / (unsigned)tiles_n);
  float2 v[RQ_IPW][RQ_CPL];
  auto load = [&](const RqIter& it) {
    const int n0 = it.nt * RQ_IN + RQ_IPW * warp, c0 = it.chunk * RQ_CH + lane;
#pragma unroll
    for (int j = 0; j < RQ_IPW; ++j) {
      const int n = n0 + j;
      const T2* row = in + ((size_t)n * T + it.t) * F + chan0;
#pragma unroll
      for (int k = 0; k < RQ_CPL; ++k) {
        const int c = c0 + 32 * k;
        v[j][k] = (n < N && c < C) ? as_float2(row[c]) : make_float2(0.f, 0.f);
      }
    }
  };
  RqIter it{(int)(blockIdx.x % (unsigned)tiles_n), (int)(blockIdx.x / (unsigned)tiles_n), 0};
  if (it.t < T) load(it);
  while (it.t < T) {
    const int n0 = it.nt * RQ_IN, c0 = it.chunk * RQ_CH, t = it.t;
#pragma unroll
    for (int k = 0; k < RQ_CPL; ++k) {
      const int c = c0 + lane + 32 * k;
      const float g = (gains && c < C) ? gains[c] : gain;
      uint32_t w4 = 0;
#pragma unroll
      for (int j = 0; j < RQ_IPW; ++j) w4 |= ((quant4(v[j][k].x, g, lo) << 4) | quant4(v[j][k].y, g, lo)) << (8 * j);
      *reinterpret_cast<uint32_t*>(&tile[lane + 32 * k][RQ_IPW * warp]) = w4;
    }
    __syncthreads();
    RqIter nx = it;
    nx.next(chunks, tiles_n, dnt, dt);
    if (nx.t < T) load(nx);  // next chunk's loads in flight during the writes
    // write: 128 channel rows x 32 input bytes, as 32-bit words where the row allows
    if (words) {
      for (int w = tid; w < RQ_CH * (RQ_IN / 4); w += RQ_NT) {
        const int cr = w / (RQ_IN / 4), nw = (w % (RQ_IN / 4)) * 4;
        if (c0 + cr < C && n0 + nw < N)
          *reinterpret_cast<uint32_t*>(out + ((size_t)t * C + c0 + cr) * N + n0 + nw) =
              *reinterpret_cast<const uint32_t*>(&tile[cr][nw]);
      }
    } else {
      for (int e = tid; e < RQ_CH * RQ_IN; e += RQ_NT) {
        const int cr = e / RQ_IN, nn = e % RQ_IN;
        if (c0 + cr < C && n0 + nn < N) out[((size_t)t * C + c0 + cr) * N + n0 + nn] = tile[cr][nn];
      }
    }
    __syncthreads();
    it = nx;
  }
}

}  // namespace

cudaError_t launch_requant(const void* d_in, int in_type, int N, int T, int F, int chan0, int C, float gain,
                           const float* d_gains, int symmetric, uint8_t* d_out, cudaStream_t st) {
  if ((long long)N * T * C == 0) return cudaSuccess;
  // persistent: one wave of resident blocks
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = in_type == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, requant_kernel<int2>, RQ_NT, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, requant_kernel<float2>, RQ_NT, 0);
  if (e != cudaSuccess) return e;
  const long long items = (long long)((N + RQ_IN - 1) / RQ_IN) * T;
  long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > items) blocks = items;
  const dim3 grid((unsigned)blocks);
  const int lo = symmetric ? -7 : -8;
  const bool words = (N & 3) == 0 && (reinterpret_cast<uintptr_t>(d_out) & 3) == 0;  // 32-bit stores stay aligned
  if (in_type == 0)
    requant_kernel<int2><<<grid, RQ_NT, 0, st>>>(static_cast<const int2*>(d_in), N, T, F, chan0, C, gain, d_gains, lo,
                                                  words, d_out);
  else
    requant_kernel<float2><<<grid, RQ_NT, 0, st>>>(static_cast<const float2*>(d_in), N, T, F, chan0, C, gain, d_gains,
                                                    lo, words, d_out);
  return cudaGetLastError();
}

}  // namespace corr
