// Total-power (autocorrelation) kernel and the dump/format kernel.
#include "corr_internal.cuh"

namespace corr {
namespace {

__device__ __forceinline__ int nib(unsigned v) { return ((int)(v & 0xF) ^ 8) - 8; }

__device__ __forceinline__ int power_of(unsigned b) {
  const int re = nib(b >> 4), im = nib(b);
  return re * re + im * im;
}

// Autocorrelations A[f][n] += sum_t |x_{f,n}(t)|^2 (Sec. 2.6: total power of selected inputs at a
// high cadence). One block of 4 warps per (channel, group of 32 inputs). Lane l of a warp reads
// the 4 inputs 4 (l % 8) .. +3 at time offset l / 8, so each warp covers 32 inputs x 4 samples per
// step and each sample byte is read once. Per-thread int32 partials are reduced over the four time
// lanes with warp shuffles, then over the 4 warps through shared memory, and added to int64.
constexpr int AW = 4;

__global__ void __launch_bounds__(AW * 32) autos_kernel(const uint8_t* __restrict__ in, int N, int C, int T,
                                                        long long* __restrict__ autos) {
  const int f = blockIdx.y;
  const int n0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane & 7, toff = lane >> 3;  // inputs n0 + 4 sub .. +3, time offset 0..3
  int acc[4] = {0, 0, 0, 0};
  long long acc64[4] = {0, 0, 0, 0};
  int since = 0;
  for (int t = warp * 4 + toff; t < T; t += AW * 4) {
    const uint8_t* row = in + ((size_t)t * C + f) * N + n0 + 4 * sub;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (n0 + 4 * sub + q < N) acc[q] += power_of(row[q]);
    if (++since == (1 << 20)) {  // int32 partials stay below 128 * 2^20
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc64[q] += acc[q];
        acc[q] = 0;
      }
      since = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long v = acc64[q] + acc[q];
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    acc64[q] = v;
  }
  __shared__ long long part[AW][32];
  if (toff == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) part[warp][4 * sub + q] = acc64[q];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int n = n0 + threadIdx.x;
    long long s = 0;
#pragma unroll
    for (int w = 0; w < AW; ++w) s += part[w][threadIdx.x];
    if (n < N) autos[(long long)f * N + n] += s;
  }
}

// Dump: out[k] = fmt(acc[k]). CI64 copies, CF32 rounds to nearest float, CF32_NORM divides by the
// sample count in double and rounds to float.
__global__ void dump_kernel(const long long* __restrict__ acc, long long n, void* __restrict__ out, int fmt,
                            long long n_samples) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long v = acc[k];
    if (fmt == CORR_FMT_CI64) {
      static_cast<long long*>(out)[k] = v;
    } else if (fmt == CORR_FMT_CF32) {
      static_cast<float*>(out)[k] = __ll2float_rn(v);
    } else {
      static_cast<float*>(out)[k] = n_samples > 0 ? __double2float_rn(__ddiv_rn(__ll2double_rn(v), (double)n_samples)) : 0.f;
    }
  }
}

}  // namespace

cudaError_t launch_autos(const Shape& s, const uint8_t* d_in, int T_blk, long long* d_autos, cudaStream_t st) {
  if (T_blk == 0) return cudaSuccess;
  dim3 grid((s.N + 31) / 32, s.C);
  autos_kernel<<<grid, AW * 32, 0, st>>>(d_in, s.N, s.C, T_blk, d_autos);
  return cudaGetLastError();
}

cudaError_t launch_dump(const long long* d_acc, long long n_elems, void* d_out, int fmt, long long n_samples,
                        cudaStream_t st) {
  if (n_elems == 0) return cudaSuccess;
  long long blocks = (n_elems + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  dump_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_acc, n_elems, d_out, fmt, n_samples);
  return cudaGetLastError();
}

}  // namespace corr
