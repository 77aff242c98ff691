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
// Thread k converts 8 inputs (chunk k % 16) of 8 samples (k / 16 + 16 j) per tile: 8-byte shared loads
// and 16-byte shared stores, both contiguous across a warp (no bank conflicts).
#include <cstring>
#include <string>

#include "corr_internal.cuh"
#include "f8_common.cuh"

namespace corr {
namespace {

constexpr int PT_THREADS = 256;
constexpr int PT_NB = 128;                 // inputs per unit
constexpr int PT_TT = 128;                 // samples per tile
constexpr int PT_RAW = PT_NB * PT_TT;      // raw tile bytes
constexpr int PT_OPR = 2 * PT_NB;          // operand rows per tile
constexpr int PT_OP = PT_OPR * PT_TT;      // operand tile bytes
constexpr int PT_STAGES = 6;
constexpr int PT_MAX_SPLIT_TILES = 256;    // <= 2048 samples per thread: 16-bit lane sums stay below 2^16
constexpr int PT_SMEM = PT_STAGES * PT_RAW + 2 * PT_OP + 1024 + 256;
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

__global__ void __launch_bounds__(PT_THREADS, 1) f8_prep_tma_kernel(const __grid_constant__ PrepTmaArgs a) {
  extern __shared__ uint8_t smem_raw_[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw_) + 1023) & ~uintptr_t(1023));
  uint8_t* raw = smem;                              // PT_STAGES x [128 t][128 n]
  uint8_t* opt = smem + PT_STAGES * PT_RAW;         // 2 x [128 t][256 r]
  uint64_t* full = reinterpret_cast<uint64_t*>(opt + 2 * PT_OP);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + PT_STAGES);
  __shared__ int red[8][16][16];                    // [warp][8-input chunk][input x (Re, Im)]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid & 15;   // 8-input chunk of the tile
  const int tq = tid >> 4;  // sample lane: samples tq + 16 j

  if (tid == 0) {
    for (int s = 0; s < PT_STAGES; ++s) ptx::mbar_init(&full[s], 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::tma_prefetch_desc(&a.in_map);
    ptx::tma_prefetch_desc(&a.op_map);
  }
  __syncthreads();

  // producer state (thread 0): next tile to load, over this CTA's units in order
  long long pu = blockIdx.x;
  int pf = 0, pib = 0, pk = 0, pk1 = 0;
  if (tid == 0 && pu < a.n_units) unit_coords(a, pu, pf, pib, pk, pk1);
  long long issued = 0;  // tiles loaded so far by this CTA
  auto issue_next = [&]() {
    if (pu >= a.n_units) return;
    const int s = (int)(issued % PT_STAGES);
    ptx::mbar_arrive_expect_tx(&full[s], PT_RAW);
    ptx::tma_load_3d(raw + s * PT_RAW, &a.in_map, &full[s], pib * PT_NB, pf, pk * PT_TT);
    ++issued;
    if (++pk == pk1) {
      pu += gridDim.x;
      if (pu < a.n_units) unit_coords(a, pu, pf, pib, pk, pk1);
    }
  };
  if (tid == 0)
    for (int s = 0; s < PT_STAGES; ++s) issue_next();

  long long consumed = 0;
  bool ok = true;
  for (long long u = blockIdx.x; u < a.n_units && ok; u += gridDim.x) {
    int f, ib, k0, k1;
    unit_coords(a, u, f, ib, k0, k1);
    const int n0 = ib * PT_NB + 8 * g;
    const int nv = a.N - n0;                           // valid inputs of this thread's chunk
    const uint32_t m0 = f8::byte_mask(nv), m1 = f8::byte_mask(nv - 4);
    // packed 16-bit lane sums: Re / Im of inputs (0, 2), (1, 3) of each 4-input word
    uint32_t sre[2][2] = {{0u, 0u}, {0u, 0u}}, sim[2][2] = {{0u, 0u}, {0u, 0u}};
    for (int k = k0; k < k1; ++k, ++consumed) {
      const int s = (int)(consumed % PT_STAGES);
      const uint32_t ph = (uint32_t)((consumed / PT_STAGES) & 1);
      const int ob = (int)(consumed & 1);
      if (tid == 0) ptx::bulk_wait_group_read<1>();  // the store of two tiles ago has read op buffer ob
      __syncthreads();
      const bool got = ptx::mbar_wait(&full[s], ph, PT_WAIT_NS);
      if (!got) *abort_flag = 1;
      if (got) {
        const uint8_t* rt = raw + s * PT_RAW;
        uint8_t* ot = opt + ob * PT_OP;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = tq + 16 * j;
          const bool tv = k * PT_TT + t < a.T;
          uint2 w = *reinterpret_cast<const uint2*>(rt + t * PT_NB + 8 * g);
          const uint32_t q0 = tv ? m0 : 0u, q1 = tv ? m1 : 0u;
          const uint4 o = make_uint4(f8::flip_hi(w.x) & q0, f8::flip_lo(w.x) & q0, f8::flip_hi(w.y) & q1,
                                     f8::flip_lo(w.y) & q1);
          *reinterpret_cast<uint4*>(ot + t * PT_OPR + 16 * g) = o;
          sre[0][0] += o.x & 0x00FF00FFu;
          sre[0][1] += (o.x >> 8) & 0x00FF00FFu;
          sim[0][0] += o.y & 0x00FF00FFu;
          sim[0][1] += (o.y >> 8) & 0x00FF00FFu;
          sre[1][0] += o.z & 0x00FF00FFu;
          sre[1][1] += (o.z >> 8) & 0x00FF00FFu;
          sim[1][0] += o.w & 0x00FF00FFu;
          sim[1][1] += (o.w >> 8) & 0x00FF00FFu;
        }
      }
      ptx::fence_proxy_async_smem();
      __syncthreads();
      if (*abort_flag) {
        ok = false;
        break;
      }
      if (tid == 0) {
        ptx::tma_store_3d(&a.op_map, opt + ob * PT_OP, 2 * ib * PT_NB, a.t_base + k * PT_TT, f);
        ptx::bulk_commit_group();
        issue_next();  // raw slot s has been read by every thread
      }
    }
    if (!ok) break;
    // per-input sums of the unit: input 8 g + 4 q + b, b = (0, 2) from [q][0], (1, 3) from [q][1]
    int v[16];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      v[2 * (4 * q + 0)] = (int)(sre[q][0] & 0xFFFF);
      v[2 * (4 * q + 2)] = (int)(sre[q][0] >> 16);
      v[2 * (4 * q + 1)] = (int)(sre[q][1] & 0xFFFF);
      v[2 * (4 * q + 3)] = (int)(sre[q][1] >> 16);
      v[2 * (4 * q + 0) + 1] = (int)(sim[q][0] & 0xFFFF);
      v[2 * (4 * q + 2) + 1] = (int)(sim[q][0] >> 16);
      v[2 * (4 * q + 1) + 1] = (int)(sim[q][1] & 0xFFFF);
      v[2 * (4 * q + 3) + 1] = (int)(sim[q][1] >> 16);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
    if (lane < 16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) red[warp][lane][j] = v[j];
    }
    __syncthreads();
    {
      // thread i: chunk i / 16, value i % 16 (input 8 (i / 16) + (i % 16) / 2, Re or Im)
      const int ch = tid >> 4, j = tid & 15;
      const int n = ib * PT_NB + 8 * ch + (j >> 1);
      long long sum = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) sum += red[w][ch][j];
      if (n < a.N && sum != 0) {
        const long long idx = ((long long)f * a.N + n) * 2 + (j & 1);
        if (a.s1) atomicAdd(reinterpret_cast<unsigned long long*>(a.s1 + idx), (unsigned long long)sum);
        if (a.s2) atomicAdd(reinterpret_cast<unsigned long long*>(a.s2 + idx), (unsigned long long)sum);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (!ok) atomicCAS(a.err, 0, 5);
    // loads still in flight land before the CTA exits; every store completes
    for (long long i = consumed; i < issued; ++i)
      ptx::mbar_wait(&full[i % PT_STAGES], (uint32_t)((i / PT_STAGES) & 1), PT_WAIT_NS);
    ptx::bulk_wait_group<0>();
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
