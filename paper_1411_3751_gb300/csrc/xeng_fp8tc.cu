// FP8 tensor-core X-engine (tcgen05, kind::f8f6f4, e4m3 operands, FP32 accumulation in TMEM).
//
// Real-valued formulation of the complex Hermitian rank-T update: per channel f the operand R_f has
// rows 2n = Re x_n and 2n + 1 = Im x_n and one column per time sample, and G_f = R_f R_f^T gives
//   Re V[a, c] = G[2a, 2c] + G[2a+1, 2c+1],   Im V[a, c] = G[2a+1, 2c] - G[2a, 2c+1]
// (V = sum_t x x^H, the X-engine product of Sec. 2.5). Integers in [-8, 7] are exact in e4m3 and
// every product is an integer of magnitude <= 64, so the FP32 tensor-core sums are exact while they
// stay below 2^24, i.e. for up to 65536 samples per flush (flushed to int64 in the epilogue).
//
// Two kernels:
//  * f8_unpack: packed bytes in[T][C][N] -> op[C][T_pad][R] e4m3 (MN-major operand, rows contiguous).
//  * f8_xeng: persistent, one CTA per SM, warp-specialised:
//      warp 0      TMA producer: 128-row x 128-sample boxes of op into a 4-stage smem ring
//      warp 1      TMEM allocator + single-thread MMA issuer (M = 128 c-side rows, N = 128 or 256
//                  a-side rows, K = 32 samples per instruction), 2 TMEM accumulators of 256 columns
//      warps 2-5   epilogue: tcgen05.ld, complex combine across lane pairs, FP32 -> int64, add to
//                  the cross / auto accumulators (each output cell is owned by one thread per launch)
//    Work item = (channel, triangle tile); tiles cover only station pairs a >= c (triangle-only
//    scheduling), with half-width tiles on the diagonal to cut wasted products.
#include <cstdio>

#include "corr_internal.cuh"
#include "ptx_sm100.cuh"

namespace corr {
namespace {

constexpr int KT = kF8Kt;
constexpr int STAGES = kF8Stages;
constexpr int A_BYTES = 128 * KT;  // 128 c-side operand rows x 128 samples
constexpr int B_ATOM = 128 * KT;   // one 128-row MN atom of the a-side operand
constexpr int B_BYTES = 2 * B_ATOM;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr uint64_t WAIT_NS = 2000000000ull;  // bounded waits: 2 s
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

// e4m3 byte of the integer value of a 4-bit two's-complement nibble (OCP FP8 E4M3: 1 sign bit,
// 4 exponent bits with bias 7, 3 mantissa bits). Small integers are normal numbers:
// |v| = 2^e (1 + m / 8).
__host__ __device__ constexpr uint32_t e4m3_of_int(int v) {
  if (v == 0) return 0u;
  const uint32_t sign = v < 0 ? 0x80u : 0u;
  const int mag = v < 0 ? -v : v;
  int e = 0;
  while ((mag >> (e + 1)) != 0) ++e;
  const uint32_t mant = (uint32_t)(((mag << 3) >> e) & 7);
  return sign | ((uint32_t)(e + 7) << 3) | mant;
}
static_assert(e4m3_of_int(1) == 0x38 && e4m3_of_int(7) == 0x4E && e4m3_of_int(-8) == 0xD0, "e4m3 encoding");

__device__ __forceinline__ uint32_t e4m3_of_nibble(uint32_t nib) {
  // table of the 16 nibble values, packed 4 per word: nibble k -> value k (k < 8) or k - 16
  constexpr uint32_t t0 = e4m3_of_int(0) | e4m3_of_int(1) << 8 | e4m3_of_int(2) << 16 | e4m3_of_int(3) << 24;
  constexpr uint32_t t1 = e4m3_of_int(4) | e4m3_of_int(5) << 8 | e4m3_of_int(6) << 16 | e4m3_of_int(7) << 24;
  constexpr uint32_t t2 = e4m3_of_int(-8) | e4m3_of_int(-7) << 8 | e4m3_of_int(-6) << 16 | e4m3_of_int(-5) << 24;
  constexpr uint32_t t3 = e4m3_of_int(-4) | e4m3_of_int(-3) << 8 | e4m3_of_int(-2) << 16 | e4m3_of_int(-1) << 24;
  const uint32_t w = (nib & 8) ? ((nib & 4) ? t3 : t2) : ((nib & 4) ? t1 : t0);
  return (w >> (8 * (nib & 3))) & 0xFF;
}

// op[f][t][r]: thread handles 16 inputs (32 operand rows) of one (f, t).
// T: valid samples, T_run: padded samples written (multiple of the stage length), T_stride: layout
// stride of op in samples per channel.
__global__ void f8_unpack_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int T_run, int T_stride, int R,
                                 bool vec, uint8_t* __restrict__ op) {
  const int G = R / 32;
  const long long total = (long long)C * T_run * G;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e % G);
    const long long ft = e / G;
    const int t = (int)(ft % T_run);
    const int f = (int)(ft / T_run);
    const int n0 = 16 * g;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (t < T && n0 < N) {
      const uint8_t* src = in + ((size_t)t * C + f) * N + n0;
      if (vec) {
        const uint4 q = *reinterpret_cast<const uint4*>(src);
        w[0] = q.x; w[1] = q.y; w[2] = q.z; w[3] = q.w;
      } else {
        for (int k = 0; k < 16; ++k)
          if (n0 + k < N) w[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
      }
    }
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t lo = 0, hi = 0;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const uint32_t byte = (w[k] >> (8 * b)) & 0xFF;
        lo |= (e4m3_of_nibble(byte >> 4) | e4m3_of_nibble(byte & 15) << 8) << (16 * b);
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const uint32_t byte = (w[k] >> (8 * (b + 2))) & 0xFF;
        hi |= (e4m3_of_nibble(byte >> 4) | e4m3_of_nibble(byte & 15) << 8) << (16 * b);
      }
      o[2 * k] = lo;
      o[2 * k + 1] = hi;
    }
    uint4* dst = reinterpret_cast<uint4*>(op + ((size_t)f * T_stride + t) * R + 32 * g);
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
  }
}

__device__ __forceinline__ void record_error(int* err, volatile int* abort_flag, int code) {
  *abort_flag = 1;
  atomicCAS(err, 0, code);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    f8_xeng_kernel(const __grid_constant__ CUtensorMap tmap, int N, int C, int npol, long long Bs, int T_run,
                   int flush_len, const F8Tile* __restrict__ tiles, int n_tiles, long long* __restrict__ cross,
                   long long* __restrict__ autos, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int P = npol * npol;
  const int n_k = T_run / KT;
  const int chunk_k = flush_len / KT;
  const long long total = (long long)n_tiles * C;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], 128);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tslot, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      ptx::tma_prefetch_desc(&tmap);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_phase[STAGES];
      bool issued[STAGES];
      for (int s = 0; s < STAGES; ++s) issued[s] = false;
      for (long long w = blockIdx.x; w < total && !*abort_flag; w += gridDim.x) {
        const int f = (int)(w / n_tiles);
        const F8Tile tl = tiles[w % n_tiles];
        const uint32_t bytes = A_BYTES + (tl.nb == 256 ? B_BYTES : B_ATOM);
        for (int ks = 0; ks < n_k; ++ks) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1, WAIT_NS)) {
            record_error(err, abort_flag, 1);
            break;
          }
          uint8_t* a_dst = smem + stage * STAGE_BYTES;
          uint8_t* b_dst = a_dst + A_BYTES;
          ptx::mbar_arrive_expect_tx(&full[stage], bytes);
          ptx::tma_load_3d(a_dst, &tmap, &full[stage], 2 * tl.c0, ks * KT, f);
          ptx::tma_load_3d(b_dst, &tmap, &full[stage], 2 * tl.a0, ks * KT, f);
          if (tl.nb == 256) ptx::tma_load_3d(b_dst + B_ATOM, &tmap, &full[stage], 2 * tl.a0 + 128, ks * KT, f);
          issued[stage] = true;
          issued_phase[stage] = phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // Copies still in flight must land before the CTA exits (normally all were consumed).
      for (int s = 0; s < STAGES; ++s)
        if (issued[s]) ptx::mbar_wait(&full[s], issued_phase[s], WAIT_NS);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id256 = ptx::idesc_f8_e4m3(128, 256, 1, 1);
      const uint32_t id128 = ptx::idesc_f8_e4m3(128, 128, 1, 1);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t use[2] = {0u, 0u};
      int acc = 0;
      bool ok = true;
      for (long long w = blockIdx.x; w < total && ok && !*abort_flag; w += gridDim.x) {
        const F8Tile tl = tiles[w % n_tiles];
        const uint32_t idesc = tl.nb == 256 ? id256 : id128;
        for (int k0 = 0; k0 < n_k && ok; k0 += chunk_k) {
          const int k1 = min(k0 + chunk_k, n_k);
          if (!ptx::mbar_wait(&tempty[acc], (use[acc] & 1) ^ 1, WAIT_NS)) {
            record_error(err, abort_flag, 2);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d = tbase + acc * ACC_COLS;
          for (int ks = k0; ks < k1; ++ks) {
            if (!ptx::mbar_wait(&full[stage], phase, WAIT_NS)) {
              record_error(err, abort_flag, 3);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a_addr = ptx::smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < KT / 32; ++kk) {
              // MN-major, 128-byte swizzle: 8 samples x 128 rows per 1024-byte atom (SBO), the
              // second 128-row atom of B at +B_ATOM (LBO).
              const uint64_t ad = ptx::smem_desc(a_addr + kk * 4096, 16, 1024, 2);
              const uint64_t bd = ptx::smem_desc(b_addr + kk * 4096, B_ATOM, 1024, 2);
              ptx::mma_f8f6f4(d, ad, bd, idesc, (ks > k0 || kk > 0) ? 1u : 0u);
            }
            ptx::mma_commit(&empty[stage]);
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          ptx::mma_commit(&tfull[acc]);
          ++use[acc];
          acc ^= 1;
        }
      }
      // all issued MMAs complete before TMEM is released
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, WAIT_NS);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const int q = warp & 3;
    const int row = 32 * q + lane;  // TMEM lane = c-side operand row
    const bool odd = (lane & 1) != 0;
    uint32_t use[2] = {0u, 0u};
    int acc = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      const int f = (int)(w / n_tiles);
      const F8Tile tl = tiles[w % n_tiles];
      const int c = tl.c0 + (row >> 1);
      const int sc = c / npol, pc = c % npol;
      for (int k0 = 0; k0 < n_k; k0 += chunk_k) {
        if (__any_sync(0xffffffffu, *abort_flag != 0)) {
          ok = false;
          break;
        }
        const bool got = ptx::mbar_wait(&tfull[acc], use[acc] & 1, WAIT_NS);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) record_error(err, abort_flag, 4);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int cc = 0; cc < tl.nb / 32; ++cc) {
          uint32_t v[32];
          ptx::tmem_ld_32x32b_x32(tbase + acc * ACC_COLS + ((uint32_t)(32 * q) << 16) + cc * 32, v);
          ptx::tmem_ld_wait();
          float recv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float send = __uint_as_float(odd ? v[j] : v[16 + j]);
            recv[j] = __shfl_xor_sync(0xffffffffu, send, 1);
          }
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            long long re, im;
            if (!odd) {  // this lane: Re_c row, partner: Im_c row; a-inputs m = 0..7 of the chunk
              re = __float2ll_rn(__uint_as_float(v[2 * m])) + __float2ll_rn(recv[2 * m + 1]);
              im = __float2ll_rn(__uint_as_float(v[2 * m + 1])) - __float2ll_rn(recv[2 * m]);
            } else {     // this lane: Im_c row, partner: Re_c row; a-inputs m = 8..15
              re = __float2ll_rn(recv[2 * m]) + __float2ll_rn(__uint_as_float(v[16 + 2 * m + 1]));
              im = __float2ll_rn(recv[2 * m + 1]) - __float2ll_rn(__uint_as_float(v[16 + 2 * m]));
            }
            const int a = tl.a0 + cc * 16 + (odd ? 8 : 0) + m;
            if (a >= N || c >= N) continue;
            const int sa = a / npol;
            if (sa < sc) continue;
            const long long b = (long long)sa * (sa + 1) / 2 + sc;
            long long* cell = cross + (((long long)f * Bs + b) * P + (a % npol) * npol + pc) * 2;
            cell[0] += re;
            cell[1] += im;
            if (a == c) autos[(long long)f * N + a] += re;
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(&tempty[acc]);
        ++use[acc];
        acc ^= 1;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

size_t f8_smem_bytes() { return SMEM_BYTES; }

cudaError_t launch_f8_unpack(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int T_stride, int R,
                             uint8_t* d_op, cudaStream_t st) {
  const long long total = (long long)s.C * T_run * (R / 32);
  if (total == 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const bool vec = (s.N % 16) == 0 && (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  f8_unpack_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_in, s.N, s.C, T_blk, T_run, T_stride, R, vec, d_op);
  return cudaGetLastError();
}

cudaError_t launch_f8_xeng(const Shape& s, const CUtensorMap* tmap, int T_run, int flush_len, const F8Tile* d_tiles,
                           int n_tiles, long long* d_cross, long long* d_autos, int* d_err, int num_sms,
                           cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(f8_xeng_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long total = (long long)n_tiles * s.C;
  if (total == 0 || T_run == 0) return cudaSuccess;
  const int grid = (int)(total < num_sms ? total : num_sms);
  f8_xeng_kernel<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(*tmap, s.N, s.C, s.npol, s.Bs, T_run, flush_len, d_tiles,
                                                         n_tiles, d_cross, d_autos, d_err);
  return cudaGetLastError();
}

int encode_op_tensor_map(CUtensorMap* map, void* d_op, int R, int T_pad, int C, std::string* err) {
  typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static encode_fn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      if (err) *err = "cuTensorMapEncodeTiled entry point unavailable";
      return -1;
    }
    fn = reinterpret_cast<encode_fn>(p);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)R, (cuuint64_t)T_pad, (cuuint64_t)C};
  const cuuint64_t strides[2] = {(cuuint64_t)R, (cuuint64_t)R * (cuuint64_t)T_pad};
  const cuuint32_t box[3] = {128, (cuuint32_t)KT, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, d_op, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed: " + std::to_string((int)r);
    return -1;
  }
  return 0;
}

}  // namespace corr
