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

constexpr int PT_CONV = 512;               // converter threads (16 warps)
constexpr int PT_CWARPS = PT_CONV / 32;
constexpr int PT_THREADS = PT_CONV + 32;   // + one producer warp (TMA loads and stores)
constexpr int PT_NB = 128;                 // inputs per unit
constexpr int PT_TT = 128;                 // samples per tile
constexpr int PT_RAW = PT_NB * PT_TT;      // raw tile bytes
constexpr int PT_OPR = 2 * PT_NB;          // operand rows per tile
constexpr int PT_OP = PT_OPR * PT_TT;      // operand tile bytes
constexpr int PT_STAGES = 6;               // raw ring
constexpr int PT_OPBUF = 3;                // operand tiles being written out
constexpr int PT_SPT = PT_TT * 16 / PT_CONV;  // samples per converter thread and tile (4)
constexpr int PT_FOLD = 4;                 // tiles per byte-lane sum (4 x 4 x 15 < 256)
constexpr int PT_MAX_SPLIT_TILES = 256;    // 1024 samples per thread: 16-bit lane sums stay below 2^16
constexpr int PT_BARS = 2 * PT_STAGES + 2 * PT_OPBUF;
constexpr int PT_SMEM = PT_STAGES * PT_RAW + PT_OPBUF * PT_OP + 1024 + 8 * PT_BARS + 64;
constexpr uint64_t PT_WAIT_NS = 2000000000ull;

struct PrepTmaArgs {
  CUtensorMap in_map;  // in[T][C][N]: dims {N, C, T}, box {128, 1, 128}
  CUtensorMap op_map;  // op[C][T_span][R_buf]: dims {R_buf, T_span, C}, box {256, 128, 1}, no swizzle
  long long* s1;
  long long* s2;
  int* err;
  int N, T, T_run, t_base;
  int n_ib;         // blocks of 128 inputs
  int n_splits;     // time splits per (channel, input block)
  int split_tiles;  // tiles per split
  long long n_units;
};

__device__ __forceinline__ void unit_coords(const PrepTmaArgs& a, long long u, int& f, int& ib, int& k0, int& k1) {
  const int sp = (int)(u % a.n_splits);
  const long long r = u / a.n_splits;
  ib = (int)(r % a.n_ib);
  f = (int)(r / a.n_ib);
  const int n_tiles = a.T_run / PT_TT;
  k0 = sp * a.split_tiles;
  k1 = min(n_tiles, k0 + a.split_tiles);
}

// Byte-lane sums (each byte at most PT_FOLD * PT_SPT * 15 < 256) into 16-bit lanes: bytes (0, 2) and (1, 3).
__device__ __forceinline__ void fold(uint32_t& acc, uint32_t (&lanes)[2]) {
  lanes[0] += acc & 0x00FF00FFu;
  lanes[1] += (acc >> 8) & 0x00FF00FFu;
  acc = 0u;
}

__device__ __forceinline__ void conv_bar_sync() { asm volatile("bar.sync 1, %0;" ::"n"(PT_CONV) : "memory"); }

// Warps 0-15 convert, warp 16 moves data. Per tile i of the CTA's sequence (its units in order, each
// unit's tiles in time order): the producer loads it into raw slot i % 6 (full[]), the converters
// read the slot (empty[] once every converter warp is done), wait until operand buffer i % 3 is free
// (opfree[]: the bulk store that last read it has finished reading), write it and signal opfull[];
// the producer then stores the buffer to the operand in global memory.
__global__ void __launch_bounds__(PT_THREADS, 1) f8_prep_tma_kernel(const __grid_constant__ PrepTmaArgs a) {
  extern __shared__ uint8_t smem_raw_[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw_) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;                              // PT_STAGES x [128 t][128 n]
  uint8_t* opt = smem + PT_STAGES * PT_RAW;         // PT_OPBUF x [128 t][256 r]
  uint64_t* full = reinterpret_cast<uint64_t*>(opt + PT_OPBUF * PT_OP);
  uint64_t* empty = full + PT_STAGES;
  uint64_t* opfull = empty + PT_STAGES;
  uint64_t* opfree = opfull + PT_OPBUF;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(opfree + PT_OPBUF);
  __shared__ int red[PT_CWARPS][16][16];            // [warp][8-input chunk][input x (Re, Im)]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < PT_STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], PT_CWARPS);
    }
    for (int b = 0; b < PT_OPBUF; ++b) {
      ptx::mbar_init(&opfull[b], PT_CWARPS);
      ptx::mbar_init(&opfree[b], 1);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();

  if (warp == PT_CWARPS) {
    // ---------------- producer: TMA loads ahead, bulk stores behind ----------------
    if (lane == 0) {
      ptx::tma_prefetch_desc(&a.in_map);
      ptx::tma_prefetch_desc(&a.op_map);
      long long lu = blockIdx.x, su = blockIdx.x;   // units of the next load / the next store
      int lf = 0, lib = 0, lk = 0, lk1 = 0, sf = 0, sib = 0, sk = 0, sk1 = 0;
      if (lu < a.n_units) unit_coords(a, lu, lf, lib, lk, lk1);
      if (su < a.n_units) unit_coords(a, su, sf, sib, sk, sk1);
      long long loaded = 0, stored = 0;
      bool ok = true;
      auto load_next = [&]() -> bool {  // false on a timeout
        if (lu >= a.n_units) return true;
        const int s = (int)(loaded % PT_STAGES);
        if (loaded >= PT_STAGES &&
            !ptx::mbar_wait(&empty[s], (uint32_t)(((loaded / PT_STAGES) - 1) & 1), PT_WAIT_NS))
          return false;
        ptx::mbar_arrive_expect_tx(&full[s], PT_RAW);
        ptx::tma_load_3d(raw + s * PT_RAW, &a.in_map, &full[s], lib * PT_NB, lf, lk * PT_TT);
        ++loaded;
        if (++lk == lk1) {
          lu += gridDim.x;
          if (lu < a.n_units) unit_coords(a, lu, lf, lib, lk, lk1);
        }
        return true;
      };
      for (int s = 0; s < PT_STAGES && ok; ++s) ok = load_next();
      while (ok && su < a.n_units) {
        const int b = (int)(stored % PT_OPBUF);
        if (!ptx::mbar_wait(&opfull[b], (uint32_t)((stored / PT_OPBUF) & 1), PT_WAIT_NS) || *abort_flag) {
          ok = false;
          break;
        }
        ptx::tma_store_3d(&a.op_map, opt + b * PT_OP, 2 * sib * PT_NB, a.t_base + sk * PT_TT, sf);
        ptx::bulk_commit_group();
        ++stored;
        if (++sk == sk1) {
          su += gridDim.x;
          if (su < a.n_units) unit_coords(a, su, sf, sib, sk, sk1);
        }
        ok = load_next();
        // all but the two newest stores have read their buffers: the tile stored - 3 frees its buffer
        ptx::bulk_wait_group_read<PT_OPBUF - 1>();
        if (stored >= PT_OPBUF) ptx::mbar_arrive(&opfree[(stored - PT_OPBUF) % PT_OPBUF]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicCAS(a.err, 0, 5);
      }
      // loads in flight land before the CTA exits; every store completes
      for (long long i = stored; i < loaded; ++i)
        ptx::mbar_wait(&full[i % PT_STAGES], (uint32_t)((i / PT_STAGES) & 1), PT_WAIT_NS);
      ptx::bulk_wait_group<0>();
    }
  } else {
    // ---------------- converters ----------------
    // Every converter warp walks every tile and every unit end (the named barrier below needs all
    // of them); after an abort the waits are skipped and nothing is converted or added.
    const int g = tid & 15;   // 8-input chunk of the tile
    const int tq = tid >> 4;  // sample lane: samples tq + 32 j
    long long consumed = 0;
    for (long long u = blockIdx.x; u < a.n_units; u += gridDim.x) {
      int f, ib, k0, k1;
      unit_coords(a, u, f, ib, k0, k1);
      const int nv = a.N - (ib * PT_NB + 8 * g);  // valid inputs of this thread's chunk
      const bool inputs_full = nv >= 8;
      const uint32_t m0 = f8::byte_mask(nv), m1 = f8::byte_mask(nv - 4);
      // per 4-input word (Re 0-3, Im 0-3, Re 4-7, Im 4-7): byte-lane sums, and 16-bit lane sums of
      // inputs (0, 2) and (1, 3)
      uint32_t acc[4] = {0u, 0u, 0u, 0u};
      uint32_t lanes[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
      for (int k = k0; k < k1; ++k, ++consumed) {
        const int s = (int)(consumed % PT_STAGES);
        const int b = (int)(consumed % PT_OPBUF);
        bool got = !*abort_flag && ptx::mbar_wait(&full[s], (uint32_t)((consumed / PT_STAGES) & 1), PT_WAIT_NS);
        if (got && consumed >= PT_OPBUF)
          got = ptx::mbar_wait(&opfree[b], (uint32_t)(((consumed / PT_OPBUF) - 1) & 1), PT_WAIT_NS);
        got = __all_sync(0xffffffffu, got);
        if (!got && lane == 0 && !*abort_flag) {
          *abort_flag = 1;
          atomicCAS(a.err, 0, 6);
        }
        if (got) {
          const uint8_t* rt = raw + s * PT_RAW + 8 * g;
          uint8_t* ot = opt + b * PT_OP + 16 * g;
          if (inputs_full && (k + 1) * PT_TT <= a.T) {
#pragma unroll
            for (int j = 0; j < PT_SPT; ++j) {
              const int t = tq + 32 * j;
              const uint2 w = *reinterpret_cast<const uint2*>(rt + t * PT_NB);
              const uint4 o = make_uint4(f8::flip_hi(w.x), f8::flip_lo(w.x), f8::flip_hi(w.y), f8::flip_lo(w.y));
              *reinterpret_cast<uint4*>(ot + t * PT_OPR) = o;
              acc[0] += o.x;
              acc[1] += o.y;
              acc[2] += o.z;
              acc[3] += o.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < PT_SPT; ++j) {
              const int t = tq + 32 * j;
              const bool tv = k * PT_TT + t < a.T;
              const uint2 w = *reinterpret_cast<const uint2*>(rt + t * PT_NB);
              const uint32_t q0 = tv ? m0 : 0u, q1 = tv ? m1 : 0u;
              const uint4 o = make_uint4(f8::flip_hi(w.x) & q0, f8::flip_lo(w.x) & q0, f8::flip_hi(w.y) & q1,
                                         f8::flip_lo(w.y) & q1);
              *reinterpret_cast<uint4*>(ot + t * PT_OPR) = o;
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
          ptx::fence_proxy_async_smem();  // the operand tile is read by the bulk store (async proxy)
        }
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&empty[s]);
          ptx::mbar_arrive(&opfull[b]);
        }
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
      conv_bar_sync();
      if (tid < 256 && !*abort_flag) {
        // thread i: chunk i / 16, value i % 16 (input 8 (i / 16) + (i % 16) / 2, Re or Im)
        const int ch = tid >> 4, j = tid & 15;
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
      conv_bar_sync();
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
  return s.N % 16 == 0 && s.N >= PT_NB && T_blk >= PT_TT && reinterpret_cast<uintptr_t>(d_in) % 16 == 0;
}

int encode_op_store_map(CUtensorMap* map, void* d_op, int R, int T_span, int C, std::string* err) {
  encode_fn_t fn = pt_encode_fn();
  if (!fn) {
    if (err) *err = "cuTensorMapEncodeTiled entry point unavailable";
    return -1;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)R, (cuuint64_t)T_span, (cuuint64_t)C};
  const cuuint64_t strides[2] = {(cuuint64_t)R, (cuuint64_t)R * (cuuint64_t)T_span};
  const cuuint32_t box[3] = {(cuuint32_t)PT_OPR, (cuuint32_t)PT_TT, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, d_op, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled (operand store) failed: " + std::to_string((int)r);
    return -1;
  }
  return 0;
}

cudaError_t launch_f8_prep_tma(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int t_base,
                               const CUtensorMap& op_store_map, long long* d_s1, long long* d_s2, int* d_err,
                               int max_ctas, cudaStream_t st) {
  if (T_run == 0) return cudaSuccess;
  cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(f8_prep_tma_kernel), PT_SMEM);
  if (e != cudaSuccess) return e;
  PrepTmaArgs a;
  std::memset(&a, 0, sizeof(a));
  encode_fn_t fn = pt_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)s.N, (cuuint64_t)s.C, (cuuint64_t)T_blk};
  const cuuint64_t strides[2] = {(cuuint64_t)s.N, (cuuint64_t)s.N * (cuuint64_t)s.C};
  const cuuint32_t box[3] = {(cuuint32_t)PT_NB, 1, (cuuint32_t)PT_TT};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (fn(&a.in_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(d_in), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  a.op_map = op_store_map;
  a.s1 = d_s1;
  a.s2 = d_s2;
  a.err = d_err;
  a.N = s.N;
  a.T = T_blk;
  a.T_run = T_run;
  a.t_base = t_base;
  a.n_ib = (s.N + PT_NB - 1) / PT_NB;
  const int n_tiles = T_run / PT_TT;
  a.n_splits = (n_tiles + PT_MAX_SPLIT_TILES - 1) / PT_MAX_SPLIT_TILES;
  a.split_tiles = (n_tiles + a.n_splits - 1) / a.n_splits;
  a.n_units = (long long)s.C * a.n_ib * a.n_splits;
  const long long grid = a.n_units < max_ctas ? a.n_units : max_ctas;
  f8_prep_tma_kernel<<<(unsigned)grid, PT_THREADS, PT_SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace corr
