// Fused FP8 tensor-core X-engine: the 4+4-bit operand build happens inside the persistent kernel,
// so the e4m3 operand never travels through HBM. Operand encoding, row order and epilogue:
// f8_common.cuh. Requires N % 16 == 0 and a 16-byte aligned input (TMA strides); the context falls
// back to the two-pass path otherwise.
//
// Work item = (channel, triangle tile): c-side block of 64 inputs (M = 128 rows) x a-side span of
// 128 or 64 inputs (N = 256 or 128 rows) with a >= c (triangle-only scheduling). Per CTA (one per
// SM, persistent), per stage of 128 samples:
//   warp 0       TMA producer: raw packed bytes in[t][f][n0 .. n0+63] of the c-block and the a-span
//                (boxes of 64 inputs x 128 samples) into a 4-slot raw ring (24 KiB per slot)
//   warps 2-9    converters: raw smem -> offset e4m3 operand in the MN-major 128-byte-swizzled
//                layout of a 2-slot operand ring (48 KiB per slot); input padding and samples
//                beyond T become zero rows
//   warp 1       TMEM allocation and the single-thread MMA issuer (M = 128, N = 256 / 128, K = 32)
//   warps 10-13  epilogue: drain of one TMEM accumulator while the MMAs fill the other
#include "f8_common.cuh"

namespace corr {
namespace {

using namespace f8;

constexpr int RAW_STAGES = 4;
constexpr int OP_STAGES = 2;
constexpr int RAW_BOX = 64 * KT;            // 64 inputs x 128 samples (8 KiB)
constexpr int RAW_BYTES = 3 * RAW_BOX;      // A box + up to 2 B boxes
constexpr int CONV_WARPS = 8;
constexpr int CONV_THREADS = 32 * CONV_WARPS;
constexpr int EPI_WARPS = 4;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int FIRST_CONV_WARP = 2;
constexpr int FIRST_EPI_WARP = FIRST_CONV_WARP + CONV_WARPS;
constexpr int NUM_THREADS = 32 * (FIRST_EPI_WARP + EPI_WARPS);
constexpr int UNITS = 6;  // 16-input units per converter thread per stage (max)
constexpr int OP_OFFSET = RAW_STAGES * RAW_BYTES;                 // 96 KiB
constexpr int BAR_OFFSET = OP_OFFSET + OP_STAGES * STAGE_BYTES;   // + 96 KiB
constexpr int SMEM_BYTES = BAR_OFFSET + 1024 + 256;

static_assert(CONV_THREADS * UNITS == 512 + 1024, "unit count per stage");
static_assert(OP_OFFSET % 1024 == 0, "operand slots must be 1024-byte aligned");

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

// raw slot -> operand slot for one stage of tile (c0, a0, nb) starting at sample t0
__device__ __forceinline__ void convert_stage(int ct, int c0, int a0, int nb, int t0, int N, int T, const uint8_t* raw,
                                              uint8_t* stage) {
  uint4 r[UNITS];
  // all shared-memory loads first
#pragma unroll
  for (int j = 0; j < UNITS; ++j) {
    bool sb;
    int t, g;
    r[j] = make_uint4(0u, 0u, 0u, 0u);
    if (!unit_map(ct, j, nb, sb, t, g)) continue;
    const uint8_t* src = sb ? raw + RAW_BOX * (1 + (g >> 2)) + t * 64 + 16 * (g & 3) : raw + t * 64 + 16 * g;
    r[j] = *reinterpret_cast<const uint4*>(src);
  }
#pragma unroll
  for (int j = 0; j < UNITS; ++j) {
    bool sb;
    int t, g;
    if (!unit_map(ct, j, nb, sb, t, g)) continue;
    const int n0 = (sb ? a0 : c0) + 16 * g;
    uint4 o0 = make_uint4(0u, 0u, 0u, 0u), o1 = make_uint4(0u, 0u, 0u, 0u);
    if (t0 + t < T && n0 < N) expand16(r[j], N - n0, o0, o1);
    // MN-major, 128-byte swizzle: sample t is a 128-byte row of its 8-row atom, 16-byte chunks
    // permuted by (t mod 8); this unit covers chunks 2 (g mod 4) and 2 (g mod 4) + 1 of the row.
    uint8_t* atom = stage + (sb ? A_BYTES + (g >> 2) * B_ATOM : 0);
    uint8_t* rowp = atom + (t >> 3) * 1024 + (t & 7) * 128;
    const int ch = 2 * (g & 3);
    *reinterpret_cast<uint4*>(rowp + ((ch ^ (t & 7)) << 4)) = o0;
    *reinterpret_cast<uint4*>(rowp + (((ch + 1) ^ (t & 7)) << 4)) = o1;
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    f8_fused_kernel(const __grid_constant__ CUtensorMap raw_map, int N, int C, int T, int T_run, int npol, long long Bs,
                    int flush_len, const F8Tile* __restrict__ tiles, int n_tiles, long long* __restrict__ cross,
                    long long* __restrict__ autos, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* raw_ring = smem;
  uint8_t* op_ring = smem + OP_OFFSET;
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(smem + BAR_OFFSET);
  uint64_t* raw_empty = raw_full + RAW_STAGES;
  uint64_t* op_full = raw_empty + RAW_STAGES;
  uint64_t* op_empty = op_full + OP_STAGES;
  uint64_t* tfull = op_empty + OP_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_k = T_run / KT;
  const int chunk_k = flush_len / KT;
  const long long total = (long long)n_tiles * C;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RAW_STAGES; ++s) {
      ptx::mbar_init(&raw_full[s], 1);
      ptx::mbar_init(&raw_empty[s], CONV_THREADS);
    }
    for (int s = 0; s < OP_STAGES; ++s) {
      ptx::mbar_init(&op_full[s], CONV_THREADS);
      ptx::mbar_init(&op_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], EPI_THREADS);
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
      // ---------------- TMA producer (raw bytes) ----------------
      ptx::tma_prefetch_desc(&raw_map);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_phase[RAW_STAGES];
      bool issued[RAW_STAGES];
      for (int s = 0; s < RAW_STAGES; ++s) issued[s] = false;
      for (long long w = blockIdx.x; w < total && !*abort_flag; w += gridDim.x) {
        const int f = (int)(w / n_tiles);
        const F8Tile tl = tiles[w % n_tiles];
        const int nbox = 1 + tl.nb / 128;
        for (int ks = 0; ks < n_k; ++ks) {
          if (!ptx::mbar_wait(&raw_empty[stage], phase ^ 1, WAIT_NS)) {
            record_error(err, abort_flag, 1);
            break;
          }
          uint8_t* dst = raw_ring + stage * RAW_BYTES;
          ptx::mbar_arrive_expect_tx(&raw_full[stage], nbox * RAW_BOX);
          ptx::tma_load_3d(dst, &raw_map, &raw_full[stage], tl.c0, f, ks * KT);
          ptx::tma_load_3d(dst + RAW_BOX, &raw_map, &raw_full[stage], tl.a0, f, ks * KT);
          if (nbox == 3) ptx::tma_load_3d(dst + 2 * RAW_BOX, &raw_map, &raw_full[stage], tl.a0 + 64, f, ks * KT);
          issued[stage] = true;
          issued_phase[stage] = phase;
          if (++stage == RAW_STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      for (int s = 0; s < RAW_STAGES; ++s)
        if (issued[s]) ptx::mbar_wait(&raw_full[s], issued_phase[s], WAIT_NS);
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
            if (!ptx::mbar_wait(&op_full[stage], phase, WAIT_NS)) {
              record_error(err, abort_flag, 3);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t a_addr = ptx::smem_u32(op_ring + stage * STAGE_BYTES);
            const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < KT / 32; ++kk) {
              const uint64_t ad = ptx::smem_desc(a_addr + kk * 4096, 16, 1024, 2);
              const uint64_t bd = ptx::smem_desc(b_addr + kk * 4096, B_ATOM, 1024, 2);
              ptx::mma_f8f6f4(d, ad, bd, idesc, (ks > k0 || kk > 0) ? 1u : 0u);
            }
            ptx::mma_commit(&op_empty[stage]);
            if (++stage == OP_STAGES) {
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
  } else if (warp < FIRST_EPI_WARP) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 32 * FIRST_CONV_WARP;
    int rs = 0, os = 0;
    uint32_t rph = 0, oph = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      const F8Tile tl = tiles[w % n_tiles];
      for (int ks = 0; ks < n_k; ++ks) {
        if (*abort_flag) {
          ok = false;
          break;
        }
        if (!ptx::mbar_wait(&raw_full[rs], rph, WAIT_NS) || !ptx::mbar_wait(&op_empty[os], oph ^ 1, WAIT_NS)) {
          record_error(err, abort_flag, 5);
          ok = false;
          break;
        }
        convert_stage(ct, tl.c0, tl.a0, tl.nb, ks * KT, N, T, raw_ring + rs * RAW_BYTES, op_ring + os * STAGE_BYTES);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ptx::mbar_arrive(&op_full[os]);
        ptx::mbar_arrive(&raw_empty[rs]);
        if (++rs == RAW_STAGES) {
          rs = 0;
          rph ^= 1;
        }
        if (++os == OP_STAGES) {
          os = 0;
          oph ^= 1;
        }
      }
    }
  } else {
    // ---------------- epilogue ----------------
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
  if (warp == 1) ptx::tmem_dealloc(tbase, TMEM_COLS);
}

}  // namespace

bool f8_fused_supported(const Shape& s, const void* d_in, int T_blk) {
  return (s.N % 16) == 0 && s.N >= 64 && T_blk >= KT && (reinterpret_cast<uintptr_t>(d_in) % 16) == 0;
}

cudaError_t launch_f8_fused(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const F8Tile* d_tiles,
                            int n_tiles, long long* d_cross, long long* d_autos, int* d_err, int num_sms,
                            cudaStream_t st) {
  {
    const cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(f8_fused_kernel), SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  const long long total = (long long)n_tiles * s.C;
  const int T_run = (int)round_up(T_blk, KT);
  if (total == 0 || T_run == 0) return cudaSuccess;
  CUtensorMap map;
  std::string err;
  if (encode_input_tensor_map(&map, d_in, s.N, s.C, T_blk, &err) != 0) return cudaErrorInvalidValue;
  const int grid = (int)(total < num_sms ? total : num_sms);
  f8_fused_kernel<<<grid, NUM_THREADS, SMEM_BYTES, st>>>(map, s.N, s.C, T_blk, T_run, s.npol, s.Bs, flush_len, d_tiles,
                                                          n_tiles, d_cross, d_autos, d_err);
  return cudaGetLastError();
}

}  // namespace corr
