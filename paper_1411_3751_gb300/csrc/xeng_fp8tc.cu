// Two-pass FP8 tensor-core X-engine (tcgen05, kind::f8f6f4, e4m3 operands, FP32 accumulation in
// TMEM). Operand encoding, row order and epilogue: f8_common.cuh.
//
//  * f8_prep (f8_prep.cu): packed bytes in[T][C][N] -> op[C][T_pad][R] (offset e4m3 operand rows)
//    plus the per-input offset sums.
//  * f8_xeng: persistent, one CTA per SM, warp-specialised:
//      warp 0      TMA producer: 128-row x 128-sample boxes of op into a 4-stage smem ring
//      warp 1      TMEM allocator + single-thread MMA issuer (M = 128 c-side rows, N = 128 or 256
//                  a-side rows, K = 32 samples per instruction), 2 TMEM accumulators of 256 columns
//      warps 2-9   epilogue: drain of one accumulator while the MMAs fill the other
//    Work item = (channel, triangle tile); tiles cover only station pairs a >= c (triangle-only
//    scheduling), with half-width tiles on the diagonal to cut wasted products; arrays of at most 32
//    inputs take items of 2 or 4 channels stacked in one tile (channel groups, below).
#include <cstdio>

#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

using namespace f8;

constexpr int B_BYTES = 2 * B_ATOM;
constexpr int NUM_THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int EPI_THREADS = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

// Ring of the wide mode (tile plan 2): each item is a pair of 64-input c-blocks against one a-block
// of up to 128 inputs, both halves sharing the B operand: a stage holds A0 | A1 | B (2 atoms), 64 KB,
// and the two M = 128 MMAs per K step write TMEM columns 0 .. 255 (half 0) and 256 .. 511 (half 1),
// so the item uses both accumulators and is drained before the next one starts.
constexpr int W_STAGES = 3;
constexpr int W_STAGE_BYTES = 2 * A_BYTES + 2 * B_ATOM;
static_assert(W_STAGES * W_STAGE_BYTES <= STAGES * STAGE_BYTES, "wide ring must fit the shared memory of the default");

// Channel groups (arrays with XengArray::cgroup = g set: g = 2 for 17 .. 32 inputs, 64 operand rows per
// channel; g = 4 for at most 16 inputs, 32 rows): an item is channels f .. f + g - 1, whose rows one TMA
// box of 128 / g rows x 128 samples x g channels (64- or 32-byte swizzle, the array's tensor map)
// stacks into a 128-row tile, each channel one MN atom of the tile (16 KB / g apart). The M = 128,
// N = 128 MMA of that tile with itself yields every channel's products as its g diagonal blocks,
// which the epilogue drains (the off-diagonal blocks, across channels, are discarded). Without the
// grouping such an array fills at most a quarter (g = 2) or a sixteenth (g = 4) of each 128 x 128
// MMA, with it g times that. Only the narrow mode (WIDE false) takes such items.
template <bool WIDE>
__global__ void __launch_bounds__(NUM_THREADS, 1) f8_xeng_kernel(const __grid_constant__ XengArgs args) {
  constexpr int RING = WIDE ? W_STAGES : STAGES;
  constexpr int RING_BYTES = WIDE ? W_STAGE_BYTES : STAGE_BYTES;
  constexpr int B_OFF = WIDE ? 2 * A_BYTES : A_BYTES;  // B within a stage
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
  const int n_k = args.T_run / KT;
  const int chunk_k = args.flush_len / KT;
  const long long total = args.n_items;
  const WorkItem* __restrict__ items = args.items;
  int* err = args.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
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
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_phase[RING];
      bool issued[RING];
      for (int s = 0; s < RING; ++s) issued[s] = false;
      for (long long w = blockIdx.x; w < total && !*abort_flag; w += gridDim.x) {
        const WorkItem tl = items[w];
        const int f = tl.f;
        const CUtensorMap* tmap = &args.a[tl.array].tmap;
        const bool cp = !WIDE && args.a[tl.array].cgroup > 1;  // channel-group item
        const bool a1 = WIDE && (tl.pad & 0xFFFF) != 0;  // second c-block present
        const uint32_t bytes = cp ? (uint32_t)A_BYTES : A_BYTES * (a1 ? 2 : 1) + (tl.nb == 256 ? B_BYTES : B_ATOM);
        for (int ks = 0; ks < n_k; ++ks) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1, WAIT_NS)) {
            record_error(err, abort_flag, 1);
            break;
          }
          uint8_t* a_dst = smem + stage * RING_BYTES;
          uint8_t* b_dst = a_dst + B_OFF;
          ptx::mbar_arrive_expect_tx(&full[stage], bytes);
          if (cp) {  // channels f .. f + g - 1 (channels past C read as zeros)
            ptx::tma_load_3d(a_dst, tmap, &full[stage], 0, ks * KT, f);
          } else {
            ptx::tma_load_3d(a_dst, tmap, &full[stage], 2 * tl.c0, ks * KT, f);
            if (a1) ptx::tma_load_3d(a_dst + A_BYTES, tmap, &full[stage], 2 * tl.c0 + 128, ks * KT, f);
            ptx::tma_load_3d(b_dst, tmap, &full[stage], 2 * tl.a0, ks * KT, f);
            if (tl.nb == 256) ptx::tma_load_3d(b_dst + B_ATOM, tmap, &full[stage], 2 * tl.a0 + 128, ks * KT, f);
          }
          issued[stage] = true;
          issued_phase[stage] = phase;
          if (++stage == RING) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // Copies still in flight must land before the CTA exits (normally all were consumed).
      for (int s = 0; s < RING; ++s)
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
        const WorkItem tl = items[w];
        const int cg = WIDE ? 0 : args.a[tl.array].cgroup;
        const bool cp = cg > 1;
        // channel groups: MN-major, swizzle of 128 / cg bytes, 8 samples x 128 / cg rows per atom (SBO),
        // channel k's rows at k x 16 KB / cg (LBO), 32 samples per MMA
        const uint32_t cg_rows = cp ? 128u / (uint32_t)cg : 0u;
        const uint32_t cg_layout = cg == 4 ? 6u : 4u;  // 32- or 64-byte swizzle
        const uint32_t idesc = tl.nb == 256 ? id256 : id128;
        // wide mode, half 1: N = nb1 columns of B starting at atom b1 (0, or 1 on a diagonal pair)
        const int nb1 = WIDE ? (tl.pad & 0xFFFF) : 0;
        const uint32_t idesc1 = nb1 == 256 ? id256 : id128;
        const uint32_t b1_off = WIDE && (tl.pad >> 16) ? (uint32_t)B_ATOM : 0u;
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
            const uint32_t a_addr = ptx::smem_u32(smem + stage * RING_BYTES);
            const uint32_t b_addr = a_addr + B_OFF;
            if (cp) {  // A and B are the same tile
#pragma unroll
              for (int kk = 0; kk < KT / 32; ++kk) {
                const uint64_t dd = ptx::smem_desc(a_addr + kk * 32 * cg_rows, cg_rows * KT, 8 * cg_rows, cg_layout);
                ptx::mma_f8f6f4(d, dd, dd, id128, (ks > k0 || kk > 0) ? 1u : 0u);
              }
            } else
#pragma unroll
            for (int kk = 0; kk < KT / 32; ++kk) {
              // MN-major, 128-byte swizzle: 8 samples x 128 rows per 1024-byte atom (SBO), the
              // second 128-row atom of B at +B_ATOM (LBO).
              const uint64_t ad = ptx::smem_desc(a_addr + kk * 4096, 16, 1024, 2);
              const uint64_t bd = ptx::smem_desc(b_addr + kk * 4096, B_ATOM, 1024, 2);
              ptx::mma_f8f6f4(d, ad, bd, idesc, (ks > k0 || kk > 0) ? 1u : 0u);
              if (WIDE && nb1 > 0) {
                const uint64_t ad1 = ptx::smem_desc(a_addr + A_BYTES + kk * 4096, 16, 1024, 2);
                const uint64_t bd1 = ptx::smem_desc(b_addr + b1_off + kk * 4096, B_ATOM, 1024, 2);
                ptx::mma_f8f6f4(d + ACC_COLS, ad1, bd1, idesc1, (ks > k0 || kk > 0) ? 1u : 0u);
              }
            }
            ptx::mma_commit(&empty[stage]);
            if (++stage == RING) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          ptx::mma_commit(&tfull[acc]);
          ++use[acc];
          if (!WIDE) acc ^= 1;  // the wide mode fills both accumulators: one handoff slot
        }
      }
      // all issued MMAs complete before TMEM is released
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, WAIT_NS);
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    // two warps per TMEM lane quarter; warp half h drains the 32-column chunks h, h + 2, ...
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    uint32_t use[2] = {0u, 0u};
    int acc = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      const WorkItem it = items[w];
      const XengArray& arr = args.a[it.array];
      F8Tile tl;
      tl.c0 = it.c0;
      tl.a0 = it.a0;
      tl.nb = it.nb;
      tl.pad = 0;
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
        if (!WIDE && arr.cgroup > 1) {
          // channel h = q / (4 / g) of the group holds rows 128 h / g .. and its own columns are the
          // 32-column chunks (4 / g) h ..; a lane quarter's two warps take one chunk each (g = 4: one
          // chunk per channel, the second warp idle); the tile offsets -64 h / g map channel h's rows
          // and columns back to its inputs 0 ..
          const int qpc = 4 / arr.cgroup;  // lane quarters (and chunks) per channel
          const int h = q / qpc;
          if (half < qpc && it.f + h < arr.C) {
            F8Tile th;
            th.c0 = -(64 / arr.cgroup) * h;
            th.a0 = th.c0;
            th.nb = 128;
            th.pad = 0;
            drain_tile(tbase + acc * ACC_COLS, q, lane, qpc * h + half, 4, th, it.f + h, arr.N, arr.npol, arr.Bs,
                       arr.cross, arr.autos);
          }
        } else if (!WIDE) {
          drain_tile(tbase + acc * ACC_COLS, q, lane, half, 2, tl, it.f, arr.N, arr.npol, arr.Bs, arr.cross, arr.autos);
        } else {
          // warps 2-5 drain half 0 (c-block c0), warps 6-9 half 1 (c-block c0 + 64, a-inputs from
          // a0 + 64 on a diagonal pair); one warp per TMEM lane quarter each
          const int nb1 = it.pad & 0xFFFF;
          if (half == 0) {
            drain_tile<true>(tbase, q, lane, 0, 1, tl, it.f, arr.N, arr.npol, arr.Bs, arr.cross, arr.autos);
          } else if (nb1 > 0) {
            F8Tile t1;
            t1.c0 = it.c0 + 64;
            t1.a0 = it.a0 + ((it.pad >> 16) ? 64 : 0);
            t1.nb = nb1;
            t1.pad = 0;
            drain_tile<true>(tbase + ACC_COLS, q, lane, 0, 1, t1, it.f, arr.N, arr.npol, arr.Bs, arr.cross, arr.autos);
          }
        }
        ptx::tc_fence_before();
        ptx::mbar_arrive(&tempty[acc]);
        ++use[acc];
        if (!WIDE) acc ^= 1;
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

cudaError_t launch_f8_xeng(const XengArgs& args, int num_sms, cudaStream_t st) {
  {
    cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(f8_xeng_kernel<false>), SMEM_BYTES);
    if (e == cudaSuccess) e = set_smem_limit(reinterpret_cast<const void*>(f8_xeng_kernel<true>), SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  if (args.pair) return launch_f8_xeng_pair(args, num_sms, st);
  if (args.n_items == 0 || args.T_run == 0) return cudaSuccess;
  const int grid = (int)(args.n_items < num_sms ? args.n_items : num_sms);
  if (args.wide)
    f8_xeng_kernel<true><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(args);
  else
    f8_xeng_kernel<false><<<grid, NUM_THREADS, SMEM_BYTES, st>>>(args);
  return cudaGetLastError();
}

std::vector<F8Tile> f8_tile_plan(int N, int R, int plan) {
  std::vector<F8Tile> t;
  if (plan == 3) {  // 128 c-inputs x 128 a-inputs per item, on a pair of SMs (xeng_pair.cu)
    for (int c0 = 0; c0 < N; c0 += 128)
      for (int a0 = c0; a0 < N; a0 += 128) {
        F8Tile x;
        x.c0 = c0;
        x.a0 = a0;
        x.nb = 256;
        x.pad = 0;
        t.push_back(x);
      }
    return t;
  }
  if (plan == 2) {
    for (int c0 = 0; c0 < N; c0 += 128)
      for (int a0 = c0; a0 < N; a0 += 128) {
        F8Tile x;
        x.c0 = c0;
        x.a0 = a0;
        x.nb = R - 2 * a0 < 256 ? R - 2 * a0 : 256;
        int nb1 = 0, hi = 0;
        if (c0 + 64 < N) {
          if (a0 == c0) {  // half 1 needs only the a-inputs from a0 + 64: the second B atom
            hi = 1;
            nb1 = 2 * a0 + 256 <= R ? 128 : 0;
          } else {
            nb1 = x.nb;
          }
        }
        x.pad = nb1 | (hi << 16);
        t.push_back(x);
      }
    return t;
  }
  const int ncb = (N + 63) / 64;
  for (int cb = 0; cb < ncb; ++cb) {
    int a0 = 64 * cb;
    int nb = (plan == 1 || (cb & 1)) ? 128 : 256;
    while (a0 < N) {
      if (2 * a0 + nb > R) nb = R - 2 * a0;
      F8Tile x;
      x.c0 = 64 * cb;
      x.a0 = a0;
      x.nb = nb;
      x.pad = 0;
      t.push_back(x);
      a0 += nb / 2;
      nb = plan == 1 ? 128 : 256;
    }
  }
  return t;
}

namespace {

typedef CUresult (*encode_fn_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn_t encode_fn(std::string* err) {
  static encode_fn_t fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      if (err) *err = "cuTensorMapEncodeTiled entry point unavailable";
      return nullptr;
    }
    fn = reinterpret_cast<encode_fn_t>(p);
  }
  return fn;
}

}  // namespace

int encode_input_tensor_map(CUtensorMap* map, const void* d_in, int N, int C, int T, std::string* err) {
  encode_fn_t fn = encode_fn(err);
  if (!fn) return -1;
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)C, (cuuint64_t)T};
  const cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * (cuuint64_t)C};
  const cuuint32_t box[3] = {64, 1, (cuuint32_t)KT};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(d_in), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (input) failed: " + std::to_string((int)r);
    return -1;
  }
  return 0;
}

int encode_op_tensor_map(CUtensorMap* map, void* d_op, int R, int T_pad, int C, std::string* err, int cgroup) {
  encode_fn_t fn = encode_fn(err);
  if (!fn) return -1;
  const bool cp = cgroup > 1;
  if (cp && !((cgroup == 2 && R == 64) || (cgroup == 4 && R == 32))) {
    if (err) *err = "channel-group tensor map needs 128 / cgroup operand rows (cgroup 2 or 4)";
    return -1;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)R, (cuuint64_t)T_pad, (cuuint64_t)C};
  const cuuint64_t strides[2] = {(cuuint64_t)R, (cuuint64_t)R * (cuuint64_t)T_pad};
  // one 128-row tile per box: 128 rows of one channel (128-byte swizzle), or 128 / g rows of each of g
  // channels (swizzle of 128 / g bytes, the channel-group items)
  const cuuint32_t box[3] = {cp ? (cuuint32_t)R : 128u, (cuuint32_t)KT, cp ? (cuuint32_t)cgroup : 1u};
  const CUtensorMapSwizzle swz =
      !cp ? CU_TENSOR_MAP_SWIZZLE_128B : (cgroup == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, d_op, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled failed: " + std::to_string((int)r);
    return -1;
  }
  return 0;
}

}  // namespace corr
