// Operand build of the two-pass FP8 tensor path (the paper's CPU "unpack" stage, Sec. 2.4, done on
// the GPU): packed bytes in[T][C][N] -> op[C][T_pad][R] (offset e4m3 bytes, group row order, MN-major:
// one contiguous row of R bytes per channel and sample) plus the per-input offset sums. Streams
// through HBM. Operand encoding and row order: f8_common.cuh.
#include <cstring>

#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

using namespace f8;

// One pass over the input. A unit = 16 inputs (32 operand rows) of one channel; units are numbered
// across channels, u = f G + g (G units per channel), so that small arrays still fill every lane. Lane l of a
// warp takes unit 8 blockIdx.x + (l % 8) at time offset l / 8, so a warp reads 8 units (128 inputs,
// contiguous in [t][C][N] when N % 16 == 0) of 4 samples and the 8 warps of a block cover 32 samples
// per step; blockIdx.z splits the time range.
//  * op (if not null): op[f][t_base + t][r] for t < T_run (zero rows for t >= T and inputs >= N);
//  * s1, s2 (if not null): per-input offset sums sum_t (x + 8 + 8i) over t < T, added to both
//    (the cross-cadence and the total-power-cadence copies). Per-thread sums live in 16-bit lanes of
//    packed words (at most 15 per sample, <= 2048 samples per thread), are reduced over the four
//    time lanes of a warp with shuffles and over the warps through shared memory, then added to the
//    int64 sums with one atomic per input and block.
constexpr int PREP_ROWS_PER_THREAD_MAX = 2048;

// The build of one block (bx, bz) of the grid: bx picks 8 units, bz the time range.
__device__ __forceinline__ void prep_block(const uint8_t* __restrict__ in, int N, int C, int T, int T_run, int T_stride,
                                           int t_base, int R, int rows_per_split, int vec, uint8_t* __restrict__ op,
                                           long long* __restrict__ s1, long long* __restrict__ s2, long long bx,
                                           int bz) {
  const int G = R / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tl = lane >> 3, us = lane & 7;
  const long long unit = 8LL * bx + us;  // flattened unit
  const bool unit_ok = unit < (long long)C * G;
  const int f = unit_ok ? (int)(unit / G) : 0;
  const int g = unit_ok ? (int)(unit - (long long)f * G) : G;
  const int t_begin = bz * rows_per_split;
  const int t_end = min(T_run, t_begin + rows_per_split);
  const int n0 = 16 * g;
  const int nv = N - n0;  // valid inputs of this unit (<= 0: padding unit)
  // packed 16-bit lane sums: [word k][even / odd byte], for Re and Im
  uint32_t sre[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
  uint32_t sim[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
  if (unit_ok) {
    // 8 samples per thread per iteration, all loads issued before any conversion
    constexpr int U = 8;
    for (int t0 = t_begin + 4 * warp + tl; t0 < t_end; t0 += 32 * U) {
      uint4 w[U];
      bool live[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + 32 * u;
        w[u] = make_uint4(0u, 0u, 0u, 0u);
        live[u] = t < t_end && t < T && nv > 0;
        if (live[u]) {
          const uint8_t* src = in + ((size_t)t * C + f) * N + n0;
          if (vec == 16) {
            w[u] = __ldg(reinterpret_cast<const uint4*>(src));
          } else if (vec == 8) {  // N % 8 == 0: nv is 8 or >= 16
            const uint2 lo = __ldg(reinterpret_cast<const uint2*>(src));
            const uint2 hi = nv > 8 ? __ldg(reinterpret_cast<const uint2*>(src) + 1) : make_uint2(0u, 0u);
            w[u] = make_uint4(lo.x, lo.y, hi.x, hi.y);
          } else if (vec == 4) {  // N % 4 == 0: nv is a multiple of 4
            const uint32_t* s4 = reinterpret_cast<const uint32_t*>(src);
            w[u] = make_uint4(__ldg(s4), nv > 4 ? __ldg(s4 + 1) : 0u, nv > 8 ? __ldg(s4 + 2) : 0u,
                              nv > 12 ? __ldg(s4 + 3) : 0u);
          } else {
            uint32_t x[4] = {0u, 0u, 0u, 0u};
            for (int k = 0; k < 16; ++k)
              if (n0 + k < N) x[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
            w[u] = make_uint4(x[0], x[1], x[2], x[3]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + 32 * u;
        if (t >= t_end) continue;
        uint4 o0 = make_uint4(0u, 0u, 0u, 0u), o1 = make_uint4(0u, 0u, 0u, 0u);
        if (live[u]) expand16(w[u], nv, o0, o1);
        if (op) {
          uint4* dst = reinterpret_cast<uint4*>(op + ((size_t)f * T_stride + t_base + t) * R + 32 * g);
          dst[0] = o0;
          dst[1] = o1;
        }
        // o0 = {Re w0, Im w0, Re w1, Im w1}, o1 = {Re w2, Im w2, Re w3, Im w3} (masked, 0 if not live)
        const uint32_t re4[4] = {o0.x, o0.z, o1.x, o1.z};
        const uint32_t im4[4] = {o0.y, o0.w, o1.y, o1.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          sre[k][0] += re4[k] & 0x00FF00FFu;
          sre[k][1] += (re4[k] >> 8) & 0x00FF00FFu;
          sim[k][0] += im4[k] & 0x00FF00FFu;
          sim[k][1] += (im4[k] >> 8) & 0x00FF00FFu;
        }
      }
    }
  }
  if (!s1 && !s2) return;
  // unpack to per-input sums, input j = 4 k + byte: even bytes 0, 2 / odd bytes 1, 3
  __shared__ int part[8][8][32];  // [warp][unit][16 inputs x (Re, Im)]
  int v[32];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * (4 * k + 0)] = (int)(sre[k][0] & 0xFFFF);
    v[2 * (4 * k + 2)] = (int)(sre[k][0] >> 16);
    v[2 * (4 * k + 1)] = (int)(sre[k][1] & 0xFFFF);
    v[2 * (4 * k + 3)] = (int)(sre[k][1] >> 16);
    v[2 * (4 * k + 0) + 1] = (int)(sim[k][0] & 0xFFFF);
    v[2 * (4 * k + 2) + 1] = (int)(sim[k][0] >> 16);
    v[2 * (4 * k + 1) + 1] = (int)(sim[k][1] & 0xFFFF);
    v[2 * (4 * k + 3) + 1] = (int)(sim[k][1] >> 16);
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    v[j] += __shfl_xor_sync(0xffffffffu, v[j], 8);
    v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
  }
  if (tl == 0) {
#pragma unroll
    for (int j = 0; j < 32; ++j) part[warp][us][j] = v[j];
  }
  __syncthreads();
  // thread i: unit i / 32, value i % 32
  const int uu = threadIdx.x >> 5, j = threadIdx.x & 31;
  const long long ug = 8LL * bx + uu;
  const int fu = (int)(ug / G), gu = (int)(ug - (long long)(ug / G) * G);
  const int n = 16 * gu + (j >> 1);
  if (ug < (long long)C * G && n < N) {
    long long sum = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += part[w][uu][j];
    if (sum != 0) {
      const long long idx = ((long long)fu * N + n) * 2 + (j & 1);
      if (s1) atomicAdd(reinterpret_cast<unsigned long long*>(s1 + idx), (unsigned long long)sum);
      if (s2) atomicAdd(reinterpret_cast<unsigned long long*>(s2 + idx), (unsigned long long)sum);
    }
  }
}

__global__ void __launch_bounds__(256) f8_prep_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int T_run,
                                                      int T_stride, int t_base, int R, int rows_per_split, int vec,
                                                      uint8_t* __restrict__ op, long long* __restrict__ s1,
                                                      long long* __restrict__ s2) {
  prep_block(in, N, C, T, T_run, T_stride, t_base, R, rows_per_split, vec, op, s1, s2, blockIdx.x, blockIdx.z);
}

// Several arrays' builds in one launch (groups of sub-arrays): job i owns the linear blocks
// [blk0_i, blk0_{i+1}), gx_i unit blocks by its time split, as its own launch would lay them out.
struct PrepJob {
  const uint8_t* in;
  uint8_t* op;
  long long* s1;
  long long* s2;
  long long blk0;
  int N, C, R, T_stride, t_base, rows, gx, vec;
};
struct PrepGroupArgs {
  PrepJob job[kMaxGroupArrays];
  int n, T, T_run;
};

__global__ void __launch_bounds__(256) f8_prep_group_kernel(const __grid_constant__ PrepGroupArgs a) {
  const long long b = blockIdx.x;
  int i = 0;
  while (i + 1 < a.n && b >= a.job[i + 1].blk0) ++i;
  const PrepJob& j = a.job[i];
  const long long local = b - j.blk0;
  prep_block(j.in, j.N, j.C, a.T, a.T_run, j.T_stride, j.t_base, j.R, j.rows, j.vec, j.op, j.s1, j.s2,
             local % j.gx, (int)(local / j.gx));
}

// Widest load (16, 8 or 4 bytes, else 1) that keeps every unit's 16 input bytes aligned: the rows of
// in[T][C][N] start at multiples of N bytes.
int load_width(int N, const void* in) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(in);
  for (int w = 16; w >= 4; w /= 2)
    if (N % w == 0 && a % w == 0) return w;
  return 1;
}

// Grid of one array's build: gx blocks of 8 units by `split` time ranges of `rows` samples.
void prep_geometry(const Shape& s, int T_run, int R, long long* gx, int* split_out, int* rows_out) {
  const int G = R / 32;
  // time split: at most PREP_ROWS_PER_THREAD_MAX samples per thread (each thread takes one of 32)
  int split = 1;
  while ((long long)(T_run + split - 1) / split > 32LL * PREP_ROWS_PER_THREAD_MAX) split *= 2;
  const long long units = (long long)G * s.C;
  // enough blocks for ~7 waves at 2 blocks per SM, so the last partial wave is a small share of the
  // launch (measured at 512 inputs: 3.4 waves 0.273 ms per 8192-sample block, 6.7 waves 0.257 ms,
  // 13.5 waves 0.257 ms, 27 waves 0.265 ms)
  const long long target = 8LL * sm_count();
  while ((units + 7) / 8 * split < target && T_run / (split * 2) >= 256) split *= 2;
  const int rows = (int)round_up((T_run + split - 1) / split, 32);
  *split_out = (T_run + rows - 1) / rows;
  *rows_out = rows;
  *gx = (units + 7) / 8;
}

}  // namespace

cudaError_t launch_f8_prep_group(const PrepJobDesc* jobs, int n, int T_blk, int T_run, cudaStream_t st) {
  if (T_run == 0 || n <= 0) return cudaSuccess;
  if (n > kMaxGroupArrays) return cudaErrorInvalidValue;
  PrepGroupArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.T = T_blk;
  a.T_run = T_run;
  long long blocks = 0;
  for (int i = 0; i < n; ++i) {
    const PrepJobDesc& d = jobs[i];
    PrepJob& j = a.job[i];
    int split = 1, rows = 0;
    long long gx = 0;
    prep_geometry(d.s, T_run, d.R, &gx, &split, &rows);
    j.in = d.in;
    j.op = d.op;
    j.s1 = d.s1;
    j.s2 = d.s2;
    j.blk0 = blocks;
    j.N = d.s.N;
    j.C = d.s.C;
    j.R = d.R;
    j.T_stride = d.T_stride;
    j.t_base = d.t_base;
    j.rows = rows;
    j.gx = (int)gx;
    j.vec = load_width(d.s.N, d.in);
    blocks += gx * split;
  }
  if (blocks == 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
  f8_prep_group_kernel<<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_f8_prep(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int T_stride, int t_base, int R,
                           uint8_t* d_op, long long* d_s1, long long* d_s2, cudaStream_t st) {
  if (T_run == 0) return cudaSuccess;
  int split = 1, rows = 0;
  long long gx = 0;
  prep_geometry(s, T_run, R, &gx, &split, &rows);
  dim3 grid((unsigned)gx, 1, split);
  const int vec = load_width(s.N, d_in);
  f8_prep_kernel<<<grid, 256, 0, st>>>(d_in, s.N, s.C, T_blk, T_run, T_stride, t_base, R, rows, vec, d_op, d_s1,
                                       d_s2);
  return cudaGetLastError();
}

}  // namespace corr
