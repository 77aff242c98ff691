// Two-SM FP8 tensor-core X-engine (tile plan 3): the multiply of the two-pass path on pairs of SMs,
// tcgen05.mma.cta_group::2 with M = 256 c-side operand rows (128 in each CTA of the pair) against
// N = 256 a-side rows (B split across the pair: 128 in each CTA), K = 32 samples per instruction,
// FP32 accumulation in TMEM, drained into the int64 cross sums by the epilogue of f8_common.cuh.
//
// Work item = (channel, 128 c-inputs C0 .. C0 + 127, 128 a-inputs A0 .. A0 + 127), A0 >= C0. CTA rank
// r of the pair holds the c-side rows of inputs C0 + 64 r .. + 63 and the a-side rows of inputs
// A0 + 64 r .. + 63; its TMEM receives the products of its c-side rows with all 256 a-side rows, i.e.
// the same 128 x 256 tile (c0 = C0 + 64 r, a0 = A0, nb = 256) that tile plan 0 gives one SM. Each SM
// thus fetches 32 KB of operand per 128 samples (16 KB c-side, 16 KB a-side) for the work of plan 0's
// 48 KB: what bounds the one-SM kernel is the per-SM operand fetch.
//
// Roles (one CTA per SM, clusters of two, warp-specialised as in xeng_fp8tc.cu):
//   warp 0       TMA producer of each CTA: its c-side and a-side boxes into a 7-stage ring; both CTAs'
//                copies complete on the even CTA's `full` barrier, whose expected bytes the even CTA
//                posts for the pair;
//   warp 1       both: the pair's TMEM allocation; even CTA: the single-thread MMA issuer, committing
//                each stage to both CTAs' `empty` barriers and each accumulator to both CTAs' `tfull`;
//   warps 2-9    epilogue of each CTA: drains its 128 TMEM lanes, then frees the accumulator on the
//                even CTA's `tempty` barrier (one arrival per warp and CTA).
// Every wait is bounded (f8::WAIT_NS); a timeout sets the error word and both CTAs' abort flags.
#include <algorithm>
#include <mutex>
#include <map>

#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

using namespace f8;

constexpr int P_THREADS = 320;
constexpr int P_EPI_WARPS = 8;
// 7 stages of 32 KB: measured at 512 inputs, 128 channels, 4 x 8192 samples, the issuer waits for
// operand data in 6.5% of its cycles with 6 stages (142.6 cycles per MMA) and 0.5% with 7 (133.6)
constexpr int P_STAGES = 7;
constexpr int P_STAGE_BYTES = A_BYTES + B_ATOM;  // per CTA: 128 c-side rows + 128 a-side rows, 128 samples
constexpr int P_SMEM_BYTES = P_STAGES * P_STAGE_BYTES + 1024 + 256;
static_assert(P_SMEM_BYTES <= 227 * 1024, "the ring must fit one CTA's shared memory");

__device__ __forceinline__ void pair_error(int* err, volatile int* abort_flag, uint32_t peer_abort, int code) {
  *abort_flag = 1;
  ptx::st_shared_cluster_u32(peer_abort, 1u);
  atomicCAS(err, 0, code);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P_THREADS, 1)
    f8_xeng_pair_kernel(const __grid_constant__ XengArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + P_STAGES * P_STAGE_BYTES);
  uint64_t* empty = full + P_STAGES;
  uint64_t* tfull = empty + P_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = rank == 0;
  const long long pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;
  const int n_k = args.T_run / KT;
  const int chunk_k = args.flush_len / KT;
  const long long total = args.n_items;
  const WorkItem* __restrict__ items = args.items;
  int* err = args.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);   // the even CTA's producer (expect_tx of both CTAs' bytes)
      ptx::mbar_init(&empty[s], 1);  // the pair's commit
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], 2 * P_EPI_WARPS);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(tslot, TMEM_COLS);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // both CTAs' barriers initialised before any remote arrival or copy
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t peer_abort = ptx::mapa_shared(const_cast<int*>(abort_flag), rank ^ 1u);

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs) ----------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_phase[P_STAGES];
      bool issued[P_STAGES];
      for (int s = 0; s < P_STAGES; ++s) issued[s] = false;
      for (long long w = pair; w < total && !*abort_flag; w += n_pairs) {
        const WorkItem tl = items[w];
        const CUtensorMap* tmap = &args.a[tl.array].tmap;
        const int row_c = 2 * tl.c0 + 128 * (int)rank, row_a = 2 * tl.a0 + 128 * (int)rank;
        for (int ks = 0; ks < n_k; ++ks) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1, WAIT_NS)) {
            pair_error(err, abort_flag, peer_abort, 1);
            break;
          }
          uint8_t* a_dst = smem + stage * P_STAGE_BYTES;
          const uint32_t bar = ptx::mapa_shared(&full[stage], 0);
          if (leader) ptx::mbar_arrive_expect_tx(&full[stage], 2u * P_STAGE_BYTES);
          ptx::tma_load_3d_pair(a_dst, tmap, bar, row_c, ks * KT, tl.f);
          ptx::tma_load_3d_pair(a_dst + A_BYTES, tmap, bar, row_a, ks * KT, tl.f);
          issued[stage] = true;
          issued_phase[stage] = phase;
          if (++stage == P_STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // The even CTA's `full` barriers count both CTAs' copies: it waits for those in flight.
      if (leader)
        for (int s = 0; s < P_STAGES; ++s)
          if (issued[s]) ptx::mbar_wait(&full[s], issued_phase[s], WAIT_NS);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (even CTA) ----------------
      const uint32_t idesc = ptx::idesc_f8_e4m3(256, 256, 1, 1);
      // descriptors of stage 0, K slice 0 (MN-major, 128-byte swizzle, one 128-row atom per operand
      // and CTA, 8 samples x 128 rows per 1024 bytes = SBO); stage s, slice kk add (s * P_STAGE_BYTES +
      // kk * 4096) / 16 to the address field, which stays below 2^14 (no carry out of the field)
      const uint64_t a_desc0 = ptx::smem_desc(ptx::smem_u32(smem), 16, 1024, 2);
      const uint64_t b_desc0 = ptx::smem_desc(ptx::smem_u32(smem) + A_BYTES, B_ATOM, 1024, 2);
      int stage = 0;
      uint32_t phase = 0;
      uint32_t use[2] = {0u, 0u};
      int acc = 0;
      bool ok = true;
      for (long long w = pair; w < total && ok && !*abort_flag; w += n_pairs) {
        for (int k0 = 0; k0 < n_k && ok; k0 += chunk_k) {
          const int k1 = min(k0 + chunk_k, n_k);
          if (!ptx::mbar_wait(&tempty[acc], (use[acc] & 1) ^ 1, WAIT_NS)) {
            pair_error(err, abort_flag, peer_abort, 2);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d = tbase + acc * ACC_COLS;
          for (int ks = k0; ks < k1; ++ks) {
            if (!ptx::mbar_wait(&full[stage], phase, WAIT_NS)) {
              pair_error(err, abort_flag, peer_abort, 3);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint64_t s_off = (uint64_t)((stage * P_STAGE_BYTES) >> 4);
#pragma unroll
            for (int kk = 0; kk < KT / 32; ++kk)
              ptx::mma_f8f6f4_pair(d, a_desc0 + s_off + kk * 256, b_desc0 + s_off + kk * 256, idesc,
                                   (ks > k0 || kk > 0) ? 1u : 0u);
            ptx::mma_commit_pair(&empty[stage], 3);
            if (++stage == P_STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!ok) break;
          ptx::mma_commit_pair(&tfull[acc], 3);
          ++use[acc];
          acc ^= 1;
        }
      }
      // all issued MMAs (into both CTAs' TMEM) complete before either CTA releases it
      ptx::mma_commit_pair(drain, 3);
      ptx::mbar_wait(drain, 0, WAIT_NS);
    } else if (lane == 0) {
      ptx::mbar_wait(drain, 0, WAIT_NS);  // odd CTA: the even CTA's last commit
    }
  } else {
    // ---------------- epilogue (warps 2..9, both CTAs) ----------------
    // two warps per TMEM lane quarter; warp half h drains the 32-column chunks h, h + 2, ...
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    uint32_t use[2] = {0u, 0u};
    int acc = 0;
    bool ok = true;
    for (long long w = pair; w < total && ok; w += n_pairs) {
      const WorkItem it = items[w];
      const XengArray& arr = args.a[it.array];
      F8Tile tl;
      tl.c0 = it.c0 + 64 * (int)rank;
      tl.a0 = it.a0;
      tl.nb = 256;
      tl.pad = 0;
      for (int k0 = 0; k0 < n_k; k0 += chunk_k) {
        if (__any_sync(0xffffffffu, *abort_flag != 0)) {
          ok = false;
          break;
        }
        const bool got = ptx::mbar_wait(&tfull[acc], use[acc] & 1, WAIT_NS);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) pair_error(err, abort_flag, peer_abort, 4);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        drain_tile(tbase + acc * ACC_COLS, q, lane, half, 2, tl, it.f, arr.N, arr.npol, arr.Bs, arr.cross, arr.autos);
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive_cluster(ptx::mapa_shared(&tempty[acc], 0));
        ++use[acc];
        acc ^= 1;
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // no CTA leaves while its peer may still signal its barriers or read its operands
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc_pair(tbase, TMEM_COLS);
}

// Clusters of this kernel that fit on the device at once (cached per device).
int max_pairs() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * (unsigned)sm_count(), 1, 1);
  cfg.blockDim = dim3(P_THREADS, 1, 1);
  cfg.dynamicSmemBytes = P_SMEM_BYTES;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, f8_xeng_pair_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cache[dev] = n;
  return n;
}

}  // namespace

cudaError_t launch_f8_xeng_pair(const XengArgs& args, int num_sms, cudaStream_t st) {
  cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(f8_xeng_pair_kernel), P_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  if (args.n_items == 0 || args.T_run == 0) return cudaSuccess;
  // one pair per two SMs the launch may use (at least one pair: given a single SM it starts when a
  // second one frees), and no more pairs than fit on the GPU at once
  long long pairs = std::max<long long>(1, std::min<long long>(args.n_items, num_sms / 2));
  const int fit = max_pairs();
  if (fit > 0) pairs = std::min<long long>(pairs, fit);
  f8_xeng_pair_kernel<<<(unsigned)(2 * pairs), P_THREADS, P_SMEM_BYTES, st>>>(args);
  return cudaGetLastError();
}

}  // namespace corr
