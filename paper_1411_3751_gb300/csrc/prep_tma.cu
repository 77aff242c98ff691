// Operand build of the two-pass tensor path with TMA on both sides, for running on a few SMs beside
// the X-engine (the paper's unpack stage, Sec. 2.4, overlapped with the cross-multiply of Sec. 2.5).
//
// The plain build (f8_prep_kernel) is limited per SM by the loads a thread can keep in flight: on a
// handful of SMs it moves ~40 GB/s each, too little to keep up with an X-engine on the rest. Here one
// persistent CTA per SM streams raw tiles in with 3-D TMA loads through a deep shared-memory ring,
// converts them in shared memory, and writes the operand tiles out with TMA bulk stores:
//
//   unit  = (channel f, block of 128 inputs, time split): up to 256 tiles of 128 samples
//   tile  = raw in[t0 .. t0 + 127][f][n0 .. n0 + 127] (16 KB, zero beyond the tensor)
//           -> operand rows 2 n0 .. 2 n0 + 255 of samples t_base + t0 .. (32 KB, clipped at the
//              operand's row count), the same bytes as f8_prep_kernel writes (f8_common.cuh:
//              offset nibble u = v + 8 as e4m3, rows in groups of Re of 4 inputs then Im of the same 4;
//              zero for inputs >= N and samples >= T)
//   sums  = per-input offset sums over the unit's valid samples, reduced in the CTA, one 64-bit
//           atomic per input and unit into both cadence copies.
// Warp-specialised: one producer warp issues the TMA loads (6 raw slots ahead) and the bulk stores
// (3 operand tiles in flight); 16 converter warps meet it only at mbarriers. Converter thread k converts
// 8 inputs (chunk k % 16) of 4 samples (k / 16 + 32 j) per tile: 8-byte shared loads and 16-byte
// shared stores, both contiguous across a warp (no bank conflicts). The offset sums add the operand
// words as packed bytes (at most 15 per sample) and widen them to 16-bit lanes every 4 tiles.
#include <cstring>
#include <string>

#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

constexpr int PT_NB = 128;                 // inputs per unit
constexpr int PT_THREAD_SAMPLES = 4096;    // samples per thread and unit: 16-bit lane sums stay below 2^16
constexpr uint64_t PT_WAIT_NS = 2000000000ull;

// Two shapes of the same kernel: CONV converter threads, a ring of STAGES raw tiles of TT samples.
//  * wide  (512, 10, 128): one CTA alone on each of a few SMs (160 KB of ring);
//  * small (128, 3, 64):   about 30 KB of shared memory, so a CTA fits beside an X-engine CTA on
//                          every SM.
template <int CONV, int STAGES, int TT>
struct PrepCfg {
  static constexpr int kConv = CONV, kStages = STAGES, kTT = TT;
  static constexpr int kWarps = CONV / 32;
  static constexpr int kThreads = CONV + 32;             // + one producer warp (TMA loads)
  static constexpr int kRaw = PT_NB * TT;                // raw tile bytes
  static constexpr int kRows = CONV / 16;                // sample lanes of a tile
  static constexpr int kSpt = TT / kRows;                // samples per converter thread and tile
  static constexpr int kFold = 255 / (kSpt * 15);        // tiles per byte-lane sum (bytes stay below 256)
  static constexpr int kSplitTiles = PT_THREAD_SAMPLES / kSpt;
  static constexpr int kSmem = STAGES * kRaw + 128 + 16 * STAGES + 64;
  static_assert(TT % kRows == 0 && kFold >= 1, "tile shape");
};
using PrepWide = PrepCfg<512, 10, 128>;
using PrepSmall = PrepCfg<128, 3, 64>;

struct PrepTmaArgs {
  CUtensorMap in_map;  // in[T][C][N]: dims {N, C, T}, box {128, 1, TT}
  uint8_t* op;         // op[C][T_span][R_buf]
  long long T_span;    // operand samples per channel
  int R_buf;           // operand rows per sample
  long long* s1;
  long long* s2;
  int* err;
  int N, T, T_run, t_base;
  int n_ib;         // blocks of 128 inputs
  int n_splits;     // time splits per (channel, input block)
  int split_tiles;  // tiles per split
  long long n_units;
};

template <int TT>
__device__ __forceinline__ void unit_coords(const PrepTmaArgs& a, long long u, int& f, int& ib, int& k0, int& k1) {
  const int sp = (int)(u % a.n_splits);
  const long long r = u / a.n_splits;
  ib = (int)(r % a.n_ib);
  f = (int)(r / a.n_ib);
  const int n_tiles = a.T_run / TT;
  k0 = sp * a.split_tiles;
  k1 = min(n_tiles, k0 + a.split_tiles);
}

// Byte-lane sums (each byte at most kFold * kSpt * 15 < 256) into 16-bit lanes: bytes (0, 2) and (1, 3).
__device__ __forceinline__ void fold(uint32_t& acc, uint32_t (&lanes)[2]) {
  lanes[0] += acc & 0x00FF00FFu;
  lanes[1] += (acc >> 8) & 0x00FF00FFu;
  acc = 0u;
}

template <int CONV>
__device__ __forceinline__ void conv_bar_sync() { asm volatile("bar.sync 1, %0;" ::"n"(CONV) : "memory"); }

// Warps 0 .. kWarps - 1 convert, the last warp loads. Per tile i of the CTA's sequence (its units in order, each unit's
// tiles in time order): the producer loads it into raw slot i % PT_STAGES (full[]); the converters
// read the slot, write the operand rows straight to global memory with 16-byte stores, and release
// the slot (empty[] once every converter warp is done).
template <class P>
__global__ void __launch_bounds__(P::kThreads, 1) f8_prep_tma_kernel(const __grid_constant__ PrepTmaArgs a) {
  constexpr int PT_CONV = P::kConv, PT_CWARPS = P::kWarps, PT_STAGES = P::kStages, PT_TT = P::kTT;
  constexpr int PT_RAW = P::kRaw, PT_SPT = P::kSpt, PT_FOLD = P::kFold, PT_ROWS = P::kRows;
  extern __shared__ uint8_t smem_raw_[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw_) + 127) & ~uintptr_t(127));
  uint8_t* raw = smem;                              // PT_STAGES x [TT t][128 n]
  uint64_t* full = reinterpret_cast<uint64_t*>(raw + PT_STAGES * PT_RAW);
  uint64_t* empty = full + PT_STAGES;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + PT_STAGES);
  __shared__ int red[PT_CWARPS][16][16];            // [warp][8-input chunk][input x (Re, Im)]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < PT_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], PT_CWARPS);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();

  if (warp == PT_CWARPS) {
    // ---------------- producer: TMA loads ahead ----------------
    if (lane == 0) {
      ptx::tma_prefetch_desc(&a.in_map);
      long long lu = blockIdx.x;
      int lf = 0, lib = 0, lk = 0, lk1 = 0;
      if (lu < a.n_units) unit_coords<PT_TT>(a, lu, lf, lib, lk, lk1);
      long long loaded = 0;
      bool ok = true;
      while (ok && lu < a.n_units && !*abort_flag) {
        const int s = (int)(loaded % PT_STAGES);
        if (loaded >= PT_STAGES &&
            !ptx::mbar_wait(&empty[s], (uint32_t)(((loaded / PT_STAGES) - 1) & 1), PT_WAIT_NS)) {
          ok = false;
          break;
        }
        ptx::mbar_arrive_expect_tx(&full[s], PT_RAW);
        ptx::tma_load_3d(raw + s * PT_RAW, &a.in_map, &full[s], lib * PT_NB, lf, lk * PT_TT);
        ++loaded;
        if (++lk == lk1) {
          lu += gridDim.x;
          if (lu < a.n_units) unit_coords<PT_TT>(a, lu, lf, lib, lk, lk1);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicCAS(a.err, 0, 5);
      }
      // loads in flight land before the CTA exits (the last PT_STAGES loads; the rest were consumed)
      for (long long i = loaded > PT_STAGES ? loaded - PT_STAGES : 0; i < loaded; ++i)
        ptx::mbar_wait(&full[i % PT_STAGES], (uint32_t)((i / PT_STAGES) & 1), PT_WAIT_NS);
    }
  } else {
    // ---------------- converters ----------------
    // Every converter warp walks every tile and every unit end (the named barrier below needs all
    // of them); after an abort the waits are skipped and nothing is converted or added.
    const int g = tid & 15;   // 8-input chunk of the tile
    const int tq = tid >> 4;  // sample lane: samples tq + PT_ROWS j
    long long consumed = 0;
    for (long long u = blockIdx.x; u < a.n_units; u += gridDim.x) {
      int f, ib, k0, k1;
      unit_coords<PT_TT>(a, u, f, ib, k0, k1);
      const int nv = a.N - (ib * PT_NB + 8 * g);  // valid inputs of this thread's chunk
      const bool inputs_full = nv >= 8;
      const uint32_t m0 = f8::byte_mask(nv), m1 = f8::byte_mask(nv - 4);
      // per 4-input word (Re 0-3, Im 0-3, Re 4-7, Im 4-7): byte-lane sums, and 16-bit lane sums of
      // inputs (0, 2) and (1, 3)
      uint32_t acc[4] = {0u, 0u, 0u, 0u};
      uint32_t lanes[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
      for (int k = k0; k < k1; ++k, ++consumed) {
        const int s = (int)(consumed % PT_STAGES);
        bool got = !*abort_flag && ptx::mbar_wait(&full[s], (uint32_t)((consumed / PT_STAGES) & 1), PT_WAIT_NS);
        got = __all_sync(0xffffffffu, got);
        if (!got && lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          atomicCAS(a.err, 0, 6);
        }
        if (got) {
          const uint8_t* rt = raw + s * PT_RAW + 8 * g;
          // operand rows 2 (128 ib + 8 g) .. + 15 of sample t_base + TT k + t; chunks past R_buf are not stored
          const int r0 = 2 * (ib * PT_NB + 8 * g);
          uint8_t* ot = a.op + ((long long)f * a.T_span + a.t_base + (long long)k * PT_TT) * a.R_buf + r0;
          const bool in_rows = r0 < a.R_buf;
          if (inputs_full && (k + 1) * PT_TT <= a.T) {
#pragma unroll
            for (int j = 0; j < PT_SPT; ++j) {
              const int t = tq + PT_ROWS * j;
              const uint2 w = *reinterpret_cast<const uint2*>(rt + t * PT_NB);
              const uint4 o = make_uint4(f8::flip_hi(w.x), f8::flip_lo(w.x), f8::flip_hi(w.y), f8::flip_lo(w.y));
              if (in_rows) __stcs(reinterpret_cast<uint4*>(ot + (long long)t * a.R_buf), o);
              acc[0] += o.x;
              acc[1] += o.y;
              acc[2] += o.z;
              acc[3] += o.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < PT_SPT; ++j) {
              const int t = tq + PT_ROWS * j;
              const bool tv = k * PT_TT + t < a.T;
              const uint2 w = *reinterpret_cast<const uint2*>(rt + t * PT_NB);
              const uint32_t q0 = tv ? m0 : 0u, q1 = tv ? m1 : 0u;
              const uint4 o = make_uint4(f8::flip_hi(w.x) & q0, f8::flip_lo(w.x) & q0, f8::flip_hi(w.y) & q1,
                                         f8::flip_lo(w.y) & q1);
              if (in_rows) __stcs(reinterpret_cast<uint4*>(ot + (long long)t * a.R_buf), o);
              acc[0] += o.x;
              acc[1] += o.y;
              acc[2] += o.z;
              acc[3] += o.w;
            }
          }
          if ((k - k0) % PT_FOLD == PT_FOLD - 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) fold(acc[q], lanes[q]);
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&empty[s]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) fold(acc[q], lanes[q]);
      // per-input sums of the unit: word q = (Re 0-3, Im 0-3, Re 4-7, Im 4-7); lanes[q][0] holds
      // inputs (0, 2) of the word, lanes[q][1] inputs (1, 3); v[2 i + c] = input i of the chunk, c = Re / Im
      int v[16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int base = 4 * (q >> 1), c = q & 1;
        v[2 * (base + 0) + c] = (int)(lanes[q][0] & 0xFFFF);
        v[2 * (base + 2) + c] = (int)(lanes[q][0] >> 16);
        v[2 * (base + 1) + c] = (int)(lanes[q][1] & 0xFFFF);
        v[2 * (base + 3) + c] = (int)(lanes[q][1] >> 16);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
      if (lane < 16) {
#pragma unroll
        for (int j = 0; j < 16; ++j) red[warp][lane][j] = v[j];
      }
      conv_bar_sync<PT_CONV>();
      for (int i = tid; i < 256 && !*abort_flag; i += PT_CONV) {
        // value i: chunk i / 16, value i % 16 (input 8 (i / 16) + (i % 16) / 2, Re or Im)
        const int ch = i >> 4, j = i & 15;
        const int n = ib * PT_NB + 8 * ch + (j >> 1);
        long long sum = 0;
#pragma unroll
        for (int w = 0; w < PT_CWARPS; ++w) sum += red[w][ch][j];
        if (n < a.N && sum != 0) {
          const long long idx = ((long long)f * a.N + n) * 2 + (j & 1);
          if (a.s1) atomicAdd(reinterpret_cast<unsigned long long*>(a.s1 + idx), (unsigned long long)sum);
          if (a.s2) atomicAdd(reinterpret_cast<unsigned long long*>(a.s2 + idx), (unsigned long long)sum);
        }
      }
      conv_bar_sync<PT_CONV>();
    }
  }
  __syncthreads();
}

typedef CUresult (*encode_fn_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn_t pt_encode_fn() {
  static encode_fn_t fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<encode_fn_t>(p);
  }
  return fn;
}

}  // namespace

bool f8_prep_tma_supported(const Shape& s, const void* d_in, int T_blk) {
  return s.N % 16 == 0 && s.N >= PT_NB && T_blk >= PrepWide::kTT && reinterpret_cast<uintptr_t>(d_in) % 16 == 0;
}

namespace {

template <class P>
cudaError_t launch_prep_variant(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int t_base, uint8_t* d_op,
                                long long T_span, int R_buf, long long* d_s1, long long* d_s2, int* d_err, int max_ctas,
                                cudaStream_t st) {
  cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(f8_prep_tma_kernel<P>), P::kSmem);
  if (e != cudaSuccess) return e;
  PrepTmaArgs a;
  std::memset(&a, 0, sizeof(a));
  encode_fn_t fn = pt_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)s.N, (cuuint64_t)s.C, (cuuint64_t)T_blk};
  const cuuint64_t strides[2] = {(cuuint64_t)s.N, (cuuint64_t)s.N * (cuuint64_t)s.C};
  const cuuint32_t box[3] = {(cuuint32_t)PT_NB, 1, (cuuint32_t)P::kTT};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (fn(&a.in_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(d_in), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  a.op = d_op;
  a.T_span = T_span;
  a.R_buf = R_buf;
  a.s1 = d_s1;
  a.s2 = d_s2;
  a.err = d_err;
  a.N = s.N;
  a.T = T_blk;
  a.T_run = T_run;
  a.t_base = t_base;
  a.n_ib = (s.N + PT_NB - 1) / PT_NB;
  const int n_tiles = T_run / P::kTT;
  a.n_splits = (n_tiles + P::kSplitTiles - 1) / P::kSplitTiles;
  a.split_tiles = (n_tiles + a.n_splits - 1) / a.n_splits;
  a.n_units = (long long)s.C * a.n_ib * a.n_splits;
  const long long grid = a.n_units < max_ctas ? a.n_units : max_ctas;
  f8_prep_tma_kernel<P><<<(unsigned)grid, P::kThreads, P::kSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_f8_prep_tma(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int t_base, uint8_t* d_op,
                               long long T_span, int R_buf, long long* d_s1, long long* d_s2, int* d_err,
                               int max_ctas, bool beside_xeng, cudaStream_t st) {
  if (T_run == 0) return cudaSuccess;
  if (beside_xeng)
    return launch_prep_variant<PrepSmall>(s, d_in, T_blk, T_run, t_base, d_op, T_span, R_buf, d_s1, d_s2, d_err,
                                          max_ctas, st);
  return launch_prep_variant<PrepWide>(s, d_in, T_blk, T_run, t_base, d_op, T_span, R_buf, d_s1, d_s2, d_err,
                                       max_ctas, st);
}

}  // namespace corr
