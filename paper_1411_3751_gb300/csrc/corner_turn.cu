// Corner turn between GPUs (paper Sec. 2.3 and Fig. 2: each F-engine board holds every channel of its
// own antennas, each X-engine GPU needs every antenna of its own channels, and the network turns the
// data from one grouping to the other). With one process per GPU the exchange is an all-to-all; these
// two kernels are its local halves, byte permutations with no arithmetic:
//  * pack:   this rank's inputs [T][C][n_local] -> one contiguous block [T][C_d][n_local] per
//            destination d, in destination order (C_d = chan_bounds[d + 1] - chan_bounds[d]);
//  * unpack: the blocks received from every source s, [T][C][n_s] each in source order ->
//            [T][C][N], source s's inputs at columns input_bounds[s] .. input_bounds[s + 1] - 1.
// Every row segment is copied with 16-byte vectors when its offsets and length allow, else bytewise.
#include <string>
#include <vector>

#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int kMaxParts = 1024;

struct Bounds {
  long long b[kMaxParts + 1];
  int n;
};

__device__ __forceinline__ int find_part(const Bounds& bd, long long x) {
  int lo = 0, hi = bd.n - 1;  // largest p with b[p] <= x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bd.b[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Copy len bytes; a warp copies one segment, lane-strided.
__device__ __forceinline__ void copy_segment(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, int len,
                                             int lane, bool vec) {
  if (vec) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = lane; i < len / 16; i += 32) d[i] = s[i];
  } else {
    for (int i = lane; i < len; i += 32) dst[i] = src[i];
  }
}

// One warp per (t, c) row of the input: its n_local bytes go to the block of the channel's destination.
// rows_before[d] = T * chan_bounds[d] (rows of the blocks before d).
__global__ void ct_pack_kernel(const uint8_t* __restrict__ in, int T, int C, int n_local, const __grid_constant__ Bounds chans,
                               uint8_t* __restrict__ out, bool vec) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long rows = (long long)T * C;
  for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const long long t = r / C;
    const int c = (int)(r - t * C);
    const int d = find_part(chans, c);
    const long long c0 = chans.b[d], cd = chans.b[d + 1] - c0;
    const long long orow = (long long)T * c0 + t * cd + (c - c0);
    copy_segment(in + r * n_local, out + orow * n_local, n_local, lane, vec);
  }
}

// One warp per (source, t, c) segment: n_s bytes of source s's block go to columns input_bounds[s].. of
// output row (t, c). off_before[s] = T * C * input_bounds[s] (bytes of the blocks before s).
__global__ void ct_unpack_kernel(const uint8_t* __restrict__ in, int T, int C, int N, const __grid_constant__ Bounds inputs,
                                 uint8_t* __restrict__ out, bool vec) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long rows = (long long)T * C;
  const long long segs = rows * inputs.n;
  for (long long w = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); w < segs; w += warps) {
    const int s = (int)(w / rows);
    const long long r = w - (long long)s * rows;
    const long long n0 = inputs.b[s], ns = inputs.b[s + 1] - n0;
    copy_segment(in + rows * n0 + r * ns, out + r * N + n0, (int)ns, lane, vec);
  }
}

int ct_fail(int code, const std::string& m) {
  set_last_error(m);
  return code;
}

bool read_bounds(const int* h, int n, long long end, Bounds* bd) {
  if (!h || n < 1 || n > kMaxParts) return false;
  if (h[0] != 0 || h[n] != end) return false;
  for (int i = 0; i < n; ++i)
    if (h[i + 1] < h[i]) return false;
  for (int i = 0; i <= n; ++i) bd->b[i] = h[i];
  bd->n = n;
  return true;
}

unsigned grid_for(long long warps_needed) {
  long long blocks = (warps_needed + 7) / 8;  // 8 warps per block
  const long long cap = (long long)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" int corr_corner_turn_pack(const void* d_in, int n_time, int n_chans, int n_local, const int* chan_bounds,
                                     int n_dest, void* d_out, void* cuda_stream) {
  if (n_time < 0 || n_chans < 0 || n_local < 0)
    return ct_fail(CORR_ERR_ARG, "corr_corner_turn_pack: need n_time, n_chans, n_local >= 0");
  Bounds bd;
  if (!read_bounds(chan_bounds, n_dest, n_chans, &bd))
    return ct_fail(CORR_ERR_ARG, "corr_corner_turn_pack: chan_bounds must run 0 = b[0] <= ... <= b[n_dest] = n_chans, "
                                 "1 <= n_dest <= 1024");
  const long long rows = (long long)n_time * n_chans;
  if (rows == 0 || n_local == 0) return CORR_OK;  // nothing to move (an empty shard)
  if (!d_in || !d_out) return ct_fail(CORR_ERR_ARG, "corr_corner_turn_pack: NULL buffer");
  const bool vec = n_local % 16 == 0 && reinterpret_cast<uintptr_t>(d_in) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(d_out) % 16 == 0;
  ct_pack_kernel<<<grid_for(rows), 256, 0, (cudaStream_t)cuda_stream>>>(static_cast<const uint8_t*>(d_in), n_time,
                                                                         n_chans, n_local, bd,
                                                                         static_cast<uint8_t*>(d_out), vec);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ct_fail(CORR_ERR_CUDA, std::string("corr_corner_turn_pack: ") + cudaGetErrorString(e));
  return CORR_OK;
}

extern "C" int corr_corner_turn_unpack(const void* d_in, int n_time, int n_chans, int n_inputs, const int* input_bounds,
                                       int n_src, void* d_out, void* cuda_stream) {
  if (n_time < 0 || n_chans < 0 || n_inputs < 0)
    return ct_fail(CORR_ERR_ARG, "corr_corner_turn_unpack: need n_time, n_chans, n_inputs >= 0");
  Bounds bd;
  if (!read_bounds(input_bounds, n_src, n_inputs, &bd))
    return ct_fail(CORR_ERR_ARG, "corr_corner_turn_unpack: input_bounds must run 0 = b[0] <= ... <= b[n_src] = "
                                 "n_inputs, 1 <= n_src <= 1024");
  const long long rows = (long long)n_time * n_chans;
  if (rows == 0 || n_inputs == 0) return CORR_OK;  // nothing to move (an empty shard)
  if (!d_in || !d_out) return ct_fail(CORR_ERR_ARG, "corr_corner_turn_unpack: NULL buffer");
  bool vec = n_inputs % 16 == 0 && reinterpret_cast<uintptr_t>(d_in) % 16 == 0 &&
             reinterpret_cast<uintptr_t>(d_out) % 16 == 0;
  for (int s = 0; s <= n_src; ++s) vec = vec && input_bounds[s] % 16 == 0;
  ct_unpack_kernel<<<grid_for(rows * n_src), 256, 0, (cudaStream_t)cuda_stream>>>(
      static_cast<const uint8_t*>(d_in), n_time, n_chans, n_inputs, bd, static_cast<uint8_t*>(d_out), vec);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ct_fail(CORR_ERR_CUDA, std::string("corr_corner_turn_unpack: ") + cudaGetErrorString(e));
  return CORR_OK;
}
