// Integer tensor-core X-engine: the Gram formulation of Sec. 2.5's cross-multiply on the warp-level
// int8 MMA (mma.sync m16n8k32, s8 x s8 -> s32), the integer tensor path of the comparison.
//
// One CTA computes a 64 x 64 block of inputs (i-block >= j-block, the lower block triangle) for one
// channel: a 128 x 128 tile of the real Gram matrix G = R R^T of the operand R (rows Re x_n and
// Im x_n, K = time). Each 128-sample K-tile of raw bytes is loaded once per CTA, transposed 4 x 4 in
// registers so that four consecutive samples of one input share a 32-bit word, split into
// sign-extended Re and Im nibbles (exact: s8 holds [-8, 7]) and stored K-major in shared memory
// (16-byte chunks XOR-swizzled by row), from where ldmatrix feeds the MMA fragments.
//
// Both sides use the same row order: each group of 16 rows holds Re of 8 inputs, then Im of the same
// 8. An m16n8 accumulator fragment then gives a thread row g (Re x_i) and row g + 8 (Im x_i) against two
// columns of one 8-wide n-tile, so the thread holding the Re-column tile of inputs j also holds their
// Im-column tile: with ReRe, ReIm, ImRe, ImIm the four real sums of one pair, V_ij = x_i conj(x_j) sums
// to (ReRe + ImIm) + i (ImRe - ReIm), with no data exchange between threads. Partials are exact s32
// (|sum| <= 64 per sample, flushed at most every 65536 samples) and are added to the int64
// accumulators at each flush.
#include "corr_internal.cuh"

namespace corr {
namespace {

constexpr int NT = 256;                     // 8 warps: 2 (i) x 4 (j)
constexpr int KT = kF8Kt;                   // samples per K-tile (128)
constexpr int TILE_ROWS = 128;              // Gram rows per side (64 inputs x Re/Im)
constexpr int SIDE_BYTES = TILE_ROWS * KT;  // 16 KiB per side per stage
constexpr int STAGE_BYTES = 2 * SIDE_BYTES;
constexpr int SMEM_BYTES = 2 * STAGE_BYTES;  // two stages

// Byte offset of (row, k) in a K-major side tile: 128-byte rows, 16-byte chunks XOR-swizzled by row.
__device__ __forceinline__ int swz(int row, int k) { return row * KT + ((((k >> 4) ^ row) & 7) << 4) + (k & 15); }

// Four sign-extended 4-bit fields (one per byte, values 0..15 as two's complement nibbles) -> s8x4:
// (v ^ 8) - 8 per byte, done as ((v ^ 8) + 0x78) ^ 0x80 so that no borrow crosses a byte.
__device__ __forceinline__ uint32_t sext4x4(uint32_t nibbles) {
  return ((nibbles ^ 0x08080808u) + 0x78787878u) ^ 0x80808080u;
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Raw bytes of 4 consecutive inputs (n0 .. n0+3 of a 64-input block starting at x0) at time t.
__device__ __forceinline__ uint32_t load_word(const uint8_t* __restrict__ in, int N, int C, int f, int T, int t,
                                              int x0, int n0, bool vec) {
  if (t >= T) return 0u;
  const int n = x0 + n0;
  if (n >= N) return 0u;
  const uint8_t* row = in + ((size_t)t * C + f) * N + n;
  if (vec) return __ldg(reinterpret_cast<const unsigned*>(row));  // N % 4 == 0, aligned base: all four valid
  uint32_t w = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (n + k < N) w |= (uint32_t)__ldg(row + k) << (8 * k);
  return w;
}

__global__ void __launch_bounds__(NT, 2)
    xeng_i8mma_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int npol, long long Bs, int flush_len,
                      const int2* __restrict__ tiles, bool vec, long long* __restrict__ cross,
                      long long* __restrict__ autos) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int2 tb = tiles[blockIdx.x];
  const int f = blockIdx.y;
  const int i0 = tb.x * 64, j0 = tb.y * 64;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;  // warp covers inputs i0 + 32 wm .. +31, j0 + 16 wn .. +15
  const int P = npol * npol;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);

  // Staging items of this thread: r = 0, 1 on the i side, r = 2, 3 on the j side. Item id (0..511 per
  // side) -> word w (4 inputs) and time quad tq: bits [1:0] and [6:5] of id give w, bits [4:2] and
  // [8:7] give tq, so a warp covers 4 words x 8 time quads (16-byte row pieces when loading, 2-way
  // bank conflicts at most when storing).
  uint32_t raw[4][4];
  auto item = [&](int r, int& w, int& tq) {
    const int id = tid + NT * (r & 1);
    w = (id & 3) | (((id >> 5) & 3) << 2);
    tq = ((id >> 2) & 7) | ((id >> 7) << 3);
  };
  auto load_tile = [&](int t0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int w, tq;
      item(r, w, tq);
      const int x0 = r < 2 ? i0 : j0;
#pragma unroll
      for (int e = 0; e < 4; ++e) raw[r][e] = load_word(in, N, C, f, T, t0 + 4 * tq + e, x0, 4 * w, vec);
    }
  };
  auto store_tile = [&](int stage) {
    uint8_t* st = smem + stage * STAGE_BYTES;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int w, tq;
      item(r, w, tq);
      uint8_t* side = st + (r < 2 ? 0 : SIDE_BYTES);
      // 4 x 4 byte transpose: y[k] = input 4w+k at times 4tq .. 4tq+3
      const uint32_t lo01 = __byte_perm(raw[r][0], raw[r][1], 0x5140), hi01 = __byte_perm(raw[r][0], raw[r][1], 0x7362);
      const uint32_t lo23 = __byte_perm(raw[r][2], raw[r][3], 0x5140), hi23 = __byte_perm(raw[r][2], raw[r][3], 0x7362);
      uint32_t y[4];
      y[0] = __byte_perm(lo01, lo23, 0x5410);
      y[1] = __byte_perm(lo01, lo23, 0x7632);
      y[2] = __byte_perm(hi01, hi23, 0x5410);
      y[3] = __byte_perm(hi01, hi23, 0x7632);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int n = 4 * w + k;  // input within the 64-input block
        const uint32_t re = sext4x4((y[k] >> 4) & 0x0F0F0F0Fu), im = sext4x4(y[k] & 0x0F0F0F0Fu);
        const int row_re = (n >> 3) * 16 + (n & 7), row_im = row_re + 8;
        *reinterpret_cast<uint32_t*>(side + swz(row_re, 4 * tq)) = re;
        *reinterpret_cast<uint32_t*>(side + swz(row_im, 4 * tq)) = im;
      }
    }
  };

  int acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][b][e] = 0;

  // on a diagonal tile, warps whose inputs j all lie above their inputs i hold no stored pair: they
  // stage samples and keep the barriers but issue no MMAs
  const bool above = tb.x == tb.y && wn * 16 >= wm * 32 + 32;
  const int n_kt = (T + KT - 1) / KT;
  load_tile(0);
  store_tile(0);
  __syncthreads();
  int since_flush = 0;
  for (int kt = 0; kt < n_kt; ++kt) {
    const bool more = kt + 1 < n_kt;
    if (more) load_tile((kt + 1) * KT);
    const uint32_t sa = sbase + (kt & 1) * STAGE_BYTES, sb = sa + SIDE_BYTES;
    const int lr = lane & 7, lm = lane >> 3;
#pragma unroll
    for (int ks = 0; ks < KT / 32; ++ks) {
      if (above) break;
      uint32_t b[4][2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {  // n8 tiles 2h, 2h+1 of this warp
        const int row = wn * 32 + (2 * h + (lm >> 1)) * 8 + lr;
        const int k = ks * 32 + (lm & 1) * 16;
        ldsm_x4(sb + swz(row, k), b[2 * h][0], b[2 * h][1], b[2 * h + 1][0], b[2 * h + 1][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        uint32_t a[4];
        const int row = wm * 64 + mt * 16 + (lm & 1) * 8 + lr;
        const int k = ks * 32 + (lm >> 1) * 16;
        ldsm_x4(sa + swz(row, k), a[0], a[1], a[2], a[3]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_s8(acc[mt][nt], a, b[nt][0], b[nt][1]);
      }
    }
    if (more) store_tile((kt + 1) & 1);
    __syncthreads();
    since_flush += KT;
    if (since_flush >= flush_len || !more) {
      since_flush = 0;
      const int g = lane >> 2, q = lane & 3;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int i = i0 + wm * 32 + mt * 8 + g;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int j = j0 + wn * 16 + h * 8 + 2 * q + e;
            const int* cr = acc[mt][2 * h];     // Re_j columns: [e] = Re_i Re_j, [2 + e] = Im_i Re_j
            const int* ci = acc[mt][2 * h + 1]; // Im_j columns: [e] = Re_i Im_j, [2 + e] = Im_i Im_j
            const long long re = (long long)cr[e] + ci[2 + e];
            const long long im = (long long)cr[2 + e] - ci[e];
            if (i >= N || j >= N) continue;
            const int s_a = i / npol, s_c = j / npol;
            if (s_a < s_c) continue;
            const long long bidx = (long long)s_a * (s_a + 1) / 2 + s_c;
            long long* cell = cross + (((long long)f * Bs + bidx) * P + (i % npol) * npol + (j % npol)) * 2;
            cell[0] += re;
            cell[1] += im;
            if (i == j) autos[(long long)f * N + i] += re;
          }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0;
      }
    }
  }
}

}  // namespace

cudaError_t launch_i8mma(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const int2* d_tiles,
                         int n_tiles, long long* d_cross, long long* d_autos, cudaStream_t st) {
  if (n_tiles == 0 || T_blk == 0) return cudaSuccess;
  {
    const cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(xeng_i8mma_kernel), SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  const bool vec = (s.N & 3) == 0 && (reinterpret_cast<uintptr_t>(d_in) & 3) == 0;
  xeng_i8mma_kernel<<<dim3(n_tiles, s.C), NT, SMEM_BYTES, st>>>(d_in, s.N, s.C, T_blk, s.npol, s.Bs, flush_len,
                                                                d_tiles, vec, d_cross, d_autos);
  return cudaGetLastError();
}

}  // namespace corr
