// Fused FP8 tensor-core X-engine: 4+4-bit unpack, tcgen05 cross-multiply and int64 flush in one
// persistent kernel. Operand encoding, row order and epilogue: f8_common.cuh.
//
// Work item = (channel, triangle tile): c-side block of 64 inputs (M = 128 rows) x a-side span of
// 128 or 64 inputs (N = 256 or 128 rows) with a >= c (triangle-only scheduling).
// Warp roles (one CTA per SM, persistent):
//   warp 0      TMEM allocation and the single-thread MMA issuer (K = 32 samples per instruction)
//   warps 1-8   converters: 16-byte global loads of packed samples, two stages of look-ahead in
//               registers, flip + nibble split, stores into the MN-major 128-byte-swizzled smem
//               operand ring (4 stages of 128 samples)
//   warps 9-12  epilogue: drain of the TMEM accumulator into the int64 cross sums
// Measured slower than the two-pass path on the [T][C][N] input layout: each converter gathers
// 64-128-byte rows 64 KiB apart and the register look-ahead cannot keep enough bytes in flight.
#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

using namespace f8;

constexpr int CONV_WARPS = 8;
constexpr int CONV_THREADS = 32 * CONV_WARPS;
constexpr int EPI_WARPS = 4;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int NUM_THREADS = 32 + CONV_THREADS + EPI_THREADS;
constexpr int UNITS = 6;                   // 16-input units per converter thread per stage (max)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

static_assert(CONV_THREADS * UNITS == 512 + 1024, "unit count per stage");

struct Item {
  int f, c0, a0, nb, t0;
  bool ok;
};

__device__ __forceinline__ Item item_at(long long i, int n_k, long long total, int n_tiles, const F8Tile* tiles) {
  Item it;
  const long long w = blockIdx.x + (i / n_k) * (long long)gridDim.x;
  it.ok = w < total;
  if (!it.ok) {
    it.f = it.c0 = it.a0 = it.t0 = 0;
    it.nb = 256;
    return it;
  }
  it.f = (int)(w / n_tiles);
  const F8Tile tl = tiles[w % n_tiles];
  it.c0 = tl.c0;
  it.a0 = tl.a0;
  it.nb = tl.nb;
  it.t0 = (int)(i % n_k) * KT;
  return it;
}

// unit j of converter thread `ct`: side (A or B), local time, 16-input group
__device__ __forceinline__ bool unit_map(int ct, int j, int nb, bool& side_b, int& t, int& g) {
  const int u = ct + CONV_THREADS * j;
  if (u < 512) {
    side_b = false;
    t = u >> 2;
    g = u & 3;
    return true;
  }
  const int v = u - 512;
  const int gb = nb >> 5;  // 8 or 4 groups of 16 inputs per sample row
  if (v >= KT * gb) return false;
  side_b = true;
  t = v / gb;
  g = v - t * gb;
  return true;
}

// Loads of stage `it` for this thread (raw packed bytes; out-of-range samples read as nothing).
__device__ __forceinline__ void load_stage(const Item& it, int ct, const uint8_t* __restrict__ in, int N, int C, int T,
                                           bool vec, uint4 (&r)[UNITS]) {
#pragma unroll
  for (int j = 0; j < UNITS; ++j) {
    r[j] = make_uint4(0u, 0u, 0u, 0u);
    bool sb;
    int t, g;
    if (!it.ok || !unit_map(ct, j, it.nb, sb, t, g)) continue;
    const int ts = it.t0 + t;
    const int n0 = (sb ? it.a0 : it.c0) + 16 * g;
    if (ts >= T || n0 >= N) continue;
    const uint8_t* src = in + ((size_t)ts * C + it.f) * N + n0;
    if (vec) {
      r[j] = __ldg(reinterpret_cast<const uint4*>(src));
    } else {
      uint32_t x[4] = {0u, 0u, 0u, 0u};
      for (int k = 0; k < 16; ++k)
        if (n0 + k < N) x[k >> 2] |= (uint32_t)__ldg(src + k) << (8 * (k & 3));
      r[j] = make_uint4(x[0], x[1], x[2], x[3]);
    }
  }
}

__device__ __forceinline__ void convert_stage(const Item& it, int ct, int N, int T, const uint4 (&r)[UNITS],
                                              uint8_t* stage) {
#pragma unroll
  for (int j = 0; j < UNITS; ++j) {
    bool sb;
    int t, g;
    if (!unit_map(ct, j, it.nb, sb, t, g)) continue;
    const int n0 = (sb ? it.a0 : it.c0) + 16 * g;
    uint4 o0 = make_uint4(0u, 0u, 0u, 0u), o1 = make_uint4(0u, 0u, 0u, 0u);
    if (it.t0 + t < T && n0 < N) expand16(r[j], N - n0, o0, o1);
    // MN-major, 128-byte swizzle: sample t is a 128-byte row of its 8-row atom, 16-byte chunks
    // permuted by (t mod 8); this unit covers chunks 2 (g mod 4) and 2 (g mod 4) + 1 of the row.
    uint8_t* atom = stage + (sb ? A_BYTES + (g >> 2) * B_ATOM : 0);
    uint8_t* rowp = atom + (t >> 3) * 1024 + (t & 7) * 128;
    const int ch = 2 * (g & 3);
    *reinterpret_cast<uint4*>(rowp + (((ch) ^ (t & 7)) << 4)) = o0;
    *reinterpret_cast<uint4*>(rowp + (((ch + 1) ^ (t & 7)) << 4)) = o1;
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    f8_fused_kernel(const uint8_t* __restrict__ in, int N, int C, int T, int T_run, int npol, long long Bs,
                    int flush_len, bool vec, const F8Tile* __restrict__ tiles, int n_tiles,
                    long long* __restrict__ cross, long long* __restrict__ autos, int* __restrict__ err) {
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
  const int n_k = T_run / KT;
  const int chunk_k = flush_len / KT;
  const long long total = (long long)n_tiles * C;
  const long long my_items = total > blockIdx.x ? (total - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long my_iters = my_items * n_k;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], CONV_THREADS);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], EPI_THREADS);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(tslot, TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0) {
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
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, WAIT_NS);
    }
  } else if (warp <= CONV_WARPS) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 32;
    uint4 r0[UNITS], r1[UNITS], r2[UNITS];
    Item i0 = item_at(0, n_k, total, n_tiles, tiles);
    Item i1 = item_at(1, n_k, total, n_tiles, tiles);
    Item i2;
    i0.ok = i0.ok && 0 < my_iters;
    i1.ok = i1.ok && 1 < my_iters;
    load_stage(i0, ct, in, N, C, T, vec, r0);
    load_stage(i1, ct, in, N, C, T, vec, r1);
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    // one step: wait for a free stage, convert, publish
    auto step = [&](const Item& it, const uint4 (&r)[UNITS]) -> bool {
      if (!ptx::mbar_wait(&empty[stage], phase ^ 1, WAIT_NS)) {
        record_error(err, abort_flag, 1);
        return false;
      }
      convert_stage(it, ct, N, T, r, smem + stage * STAGE_BYTES);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ptx::mbar_arrive(&full[stage]);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
      return true;
    };
    for (long long i = 0; i < my_iters && ok; i += 3) {
      if (*abort_flag) break;
      i2 = item_at(i + 2, n_k, total, n_tiles, tiles);
      i2.ok = i2.ok && (i + 2) < my_iters;
      load_stage(i2, ct, in, N, C, T, vec, r2);
      ok = step(i0, r0);
      if (!ok || i + 1 >= my_iters) break;
      i0 = item_at(i + 3, n_k, total, n_tiles, tiles);
      i0.ok = i0.ok && (i + 3) < my_iters;
      load_stage(i0, ct, in, N, C, T, vec, r0);
      ok = step(i1, r1);
      if (!ok || i + 2 >= my_iters) break;
      i1 = item_at(i + 4, n_k, total, n_tiles, tiles);
      i1.ok = i1.ok && (i + 4) < my_iters;
      load_stage(i1, ct, in, N, C, T, vec, r1);
      ok = step(i2, r2);
    }
  } else {
    // ---------------- epilogue (warps 9..12) ----------------
    const int q = warp & 3;
    uint32_t use[2] = {0u, 0u};
    int acc = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      const int f = (int)(w / n_tiles);
      const F8Tile tl = tiles[w % n_tiles];
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
        drain_tile(tbase + acc * ACC_COLS, q, lane, 0, 1, tl, f, N, npol, Bs, cross, autos);
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
  if (warp == 0) ptx::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

cudaError_t launch_f8_fused(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const F8Tile* d_tiles,
                            int n_tiles, long long* d_cross, long long* d_autos, int* d_err, int num_sms,
                            cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(f8_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long total = (long long)n_tiles * s.C;
  const int T_run = (int)round_up(T_blk, KT);
  if (total == 0 || T_run == 0) return cudaSuccess;
  const int grid = (int)(total < num_sms ? total : num_sms);
  const bool vec = (s.N % 16) == 0 && (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
  f8_fused_kernel<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(d_in, s.N, s.C, T_blk, T_run, s.npol, s.Bs, flush_len, vec,
                                                          d_tiles, n_tiles, d_cross, d_autos, d_err);
  return cudaGetLastError();
}

}  // namespace corr
