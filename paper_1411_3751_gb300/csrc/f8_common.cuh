// Pieces shared by the two FP8 tensor-core X-engines (two-pass TMA-fed and fused): the offset
// operand encoding and the epilogue that drains one TMEM accumulator into the int64 cross sums.
//
// Operand encoding (exact). Each 4-bit two's-complement component v in [-8, 7] enters the tensor
// cores as u = v + 8 in [0, 15], i.e. the nibble with its sign bit flipped. The e4m3 bytes
// 0x00..0x0F are exactly u * 2^-9 (subnormals 0..7 and the first normal binade 8..15 share the
// spacing 2^-9), so the operand byte IS the flipped nibble. Products are u_r u_s 2^-18 and the
// FP32 TMEM sums are exact while the integer sum stays below 2^24 (225 * 65536 < 2^24, the largest
// flush period). The kernels accumulate the offset-domain visibility Vu = sum_t u_a conj(u_c)
// (u = x + 8 + 8i) and its diagonal Au = sum_t |u_a|^2; the dump maps them back with the per-input
// sums s = sum_t u (Re s, Im s):
//     V = Vu - (8 - 8i) s_a - (8 + 8i) conj(s_c) + 128 T,    A = Au - 16 (Re s + Im s) + 128 T.
//
// Operand rows per channel come in groups of 8: Re of 4 consecutive inputs, then Im of the same 4
// inputs; one column (K) per time sample. With G = R R^T the X-engine product of Sec. 2.5 is
//   Re V[a, c] = G[Re a, Re c] + G[Im a, Im c],   Im V[a, c] = G[Im a, Re c] - G[Re a, Im c].
#pragma once

#include "corr_internal.cuh"
#include "ptx_sm100.cuh"

namespace corr {
namespace f8 {

constexpr int KT = kF8Kt;          // samples per pipeline stage
constexpr int STAGES = kF8Stages;
constexpr int A_BYTES = 128 * KT;  // 128 c-side rows x 128 samples
constexpr int B_ATOM = 128 * KT;   // one 128-row MN atom of the a-side operand
constexpr int STAGE_BYTES = A_BYTES + 2 * B_ATOM;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr uint64_t WAIT_NS = 2000000000ull;  // bounded waits: 2 s

// 4 packed samples -> offset operand bytes: Re of the 4 inputs / Im of the 4 inputs.
__device__ __forceinline__ uint32_t flip_hi(uint32_t w) { return ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u; }
__device__ __forceinline__ uint32_t flip_lo(uint32_t w) { return (w & 0x0F0F0F0Fu) ^ 0x08080808u; }

// first nvalid (0..4) bytes of a word kept
__device__ __forceinline__ uint32_t byte_mask(int nvalid) {
  return nvalid >= 4 ? 0xFFFFFFFFu : (nvalid <= 0 ? 0u : (0xFFFFFFFFu >> (8 * (4 - nvalid))));
}

// 16 packed samples of inputs n0..n0+15 (nv of them valid) -> 32 operand bytes in group order.
__device__ __forceinline__ void expand16(const uint4& r, int nv, uint4& o0, uint4& o1) {
  const uint32_t m0 = byte_mask(nv), m1 = byte_mask(nv - 4), m2 = byte_mask(nv - 8), m3 = byte_mask(nv - 12);
  o0 = make_uint4(flip_hi(r.x) & m0, flip_lo(r.x) & m0, flip_hi(r.y) & m1, flip_lo(r.y) & m1);
  o1 = make_uint4(flip_hi(r.z) & m2, flip_lo(r.z) & m2, flip_hi(r.w) & m3, flip_lo(r.w) & m3);
}

// TMEM partial sum (integer * 2^-18, |integer| < 2^24) -> the integer
__device__ __forceinline__ int to_int(float x) { return __float2int_rn(x * 262144.0f); }

__device__ __forceinline__ void record_error(int* err, volatile int* abort_flag, int code) {
  *abort_flag = 1;
  atomicCAS(err, 0, code);
}

// Drain the accumulator at TMEM column `tacc` (128 lanes = c-side rows of tile tl, nb columns =
// a-side rows) into cross[f]. Called by a warp of lane quarter q; the warps sharing a quarter take
// 32-column chunks first, first + stride, ... Per chunk each thread owns 8 output cells: the lane
// holding Re c and its partner holding Im c (lane ^ 4) exchange half of their columns by shuffle,
// and all 8 loads of the old int64 values are issued before any store. With RED the sums are added
// by fire-and-forget 64-bit reductions instead (no load to wait for; exact in any order).
// Diagonal cells (a == c) are also added to autos[f][a] (offset-domain total power).
template <bool RED = false>
__device__ __forceinline__ void drain_tile(uint32_t tacc, int q, int lane, int first, int stride, const F8Tile& tl,
                                           int f, int N, int npol, long long Bs, long long* __restrict__ cross,
                                           long long* __restrict__ autos) {
  const int P = npol * npol;
  const int row = 32 * q + lane;
  const bool im_lane = (lane & 4) != 0;
  const int c = tl.c0 + 4 * (row >> 3) + (row & 3);
  const int sc = c / npol, pc = c % npol;
  const int n_chunks = tl.nb / 32;
  for (int cc = first; cc < n_chunks; cc += stride) {
    uint32_t v[32];
    ptx::tmem_ld_32x32b_x32(tacc + ((uint32_t)(32 * q) << 16) + cc * 32, v);
    ptx::tmem_ld_wait();
    // columns of the chunk: 16 a-inputs, column 8 (k / 4) + k % 4 = Re a_k, + 4 = Im a_k
    float recv[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float send = __uint_as_float(im_lane ? v[j] : v[16 + j]);
      recv[j] = __shfl_xor_sync(0xffffffffu, send, 4);
    }
    int re[8], im[8];
    long long* cell[8];
    uint32_t valid = 0u;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int jr = 8 * (m >> 2) + (m & 3), ji = jr + 4;
      if (!im_lane) {  // own row Re c; partner row Im c; a-inputs k = m
        re[m] = to_int(__uint_as_float(v[jr])) + to_int(recv[ji]);
        im[m] = to_int(__uint_as_float(v[ji])) - to_int(recv[jr]);
      } else {         // own row Im c; partner row Re c; a-inputs k = 8 + m
        re[m] = to_int(recv[jr]) + to_int(__uint_as_float(v[16 + ji]));
        im[m] = to_int(recv[ji]) - to_int(__uint_as_float(v[16 + jr]));
      }
      const int a = tl.a0 + cc * 16 + (im_lane ? 8 : 0) + m;
      cell[m] = cross;  // in-bounds placeholder for skipped cells (loaded, never stored)
      if (a < N && c < N) {
        const int sa = a / npol;
        if (sa >= sc) {
          const long long b = (long long)sa * (sa + 1) / 2 + sc;
          cell[m] = cross + (((long long)f * Bs + b) * P + (a % npol) * npol + pc) * 2;
          valid |= 1u << m;
          if (a == c) {
            if (RED)
              atomicAdd(reinterpret_cast<unsigned long long*>(autos + (long long)f * N + a), (unsigned long long)(long long)re[m]);
            else
              autos[(long long)f * N + a] += re[m];
          }
        }
      }
    }
    if (RED) {
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (valid & (1u << m)) {
          atomicAdd(reinterpret_cast<unsigned long long*>(cell[m]), (unsigned long long)(long long)re[m]);
          atomicAdd(reinterpret_cast<unsigned long long*>(cell[m]) + 1, (unsigned long long)(long long)im[m]);
        }
    } else {
      longlong2 old[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) old[m] = *reinterpret_cast<const longlong2*>(cell[m]);
#pragma unroll
      for (int m = 0; m < 8; ++m)
        if (valid & (1u << m))
          *reinterpret_cast<longlong2*>(cell[m]) = make_longlong2(old[m].x + re[m], old[m].y + im[m]);
    }
  }
}

}  // namespace f8
}  // namespace corr
