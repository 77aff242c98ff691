// Internal declarations shared by the libcorr translation units (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "corr.h"

namespace corr {

// ---------------------------------------------------------------------------------------------
// Sizes and layouts
// ---------------------------------------------------------------------------------------------
// Accumulators (int64, owned by the context):
//   cross[C][B_s][P][2]   exactly the public cross layout (corr.h), P = n_pol^2
//   autos[C][N]
// FP8 tensor path scratch (e4m3 operand, rebuilt by every corr_accumulate):
//   op[C][T_pad][R]       R = round_up(2N, 128) operand rows per channel in groups of 8 (Re of 4
//                         inputs, Im of the same 4; offset encoding of f8_common.cuh; zero beyond
//                         the last input), T_pad = round_up(T, 128) time columns (zero beyond T).
//                         Time is the contraction (K) dimension and the rows are contiguous, i.e.
//                         an MN-major operand for the tensor cores.

struct Shape {
  int N, C, T, npol;
  int S;        // stations
  long long Bs; // station pairs
  int P;        // products per pair
};

// Offset-domain correction parameters for dumps (soff == nullptr: no correction).
struct Shape2 {
  int N, npol, P;
  long long Bs;
  const long long* soff;  // [C][N][2] offset sums of the tensor path
  long long t_off;        // samples accumulated through the tensor path
  int autos;              // 1: the accumulator is autos[C][N], else cross[C][B_s][P][2]
  const long long* base;  // per station pair (cross) or input (autos): sample count at the cell's last
                          // selective reset, or nullptr if no cell was ever reset selectively
};

// FP8 path tile: c-side block of 64 inputs (128 operand rows, the MMA's M), a-side block starting
// at input a0 with nb operand rows (128 or 256, the MMA's N).
struct F8Tile {
  int c0;
  int a0;
  int nb;
  int pad;
};

// One work item of the tensor-core X-engine: a tile of one channel of one array.
struct WorkItem {
  int array, f, c0, a0, nb, pad;
};

// Per-array parameters of a tensor-core X-engine launch (one array, or a group of sub-arrays of
// different N correlated in one persistent launch).
constexpr int kMaxGroupArrays = 8;
struct XengArray {
  CUtensorMap tmap;  // operand op[C][T_span][R] (the channel-group box when cgroup is set)
  long long* cross;
  long long* autos;
  long long Bs;
  int N, npol;
  int C;       // channels (the channel-group epilogue skips channels past C)
  int cgroup;  // 0, or channels per item (2: 64 operand rows per channel, 4: 32 rows): items are
               // channels f .. f + cgroup - 1 stacked in one 128-row tile (c0 = a0 = 0, nb = 128)
};
struct XengArgs {
  XengArray a[kMaxGroupArrays];
  const WorkItem* items;
  long long n_items;
  int T_run;      // samples multiplied per item (multiple of kF8Kt)
  int flush_len;  // samples per in-chip partial sum
  int* err;
  int wide;       // items are c-block pairs of tile plan 2 (see f8_tile_plan)
  int pair;       // items are the 128 x 128-input tiles of tile plan 3, multiplied on SM pairs
};

constexpr int kF8Kt = 128;             // time samples per pipeline stage
constexpr int kF8Stages = 4;           // smem ring depth
constexpr int kF8RowAlign = 128;       // operand row padding
constexpr int kF8MaxFlush = 65536;     // FP32 TMEM partials stay exact below 2^24 = 64 * 2^18
constexpr int kF32Kt = 32;             // FP32 path time granule
constexpr int kF32MaxFlush = 65536;    // |partial| <= 128 * 65536 = 2^23 < 2^24
constexpr int kDefaultFlushF8 = 65536;
constexpr int kDefaultFlushF32 = 65536;
constexpr unsigned long long kMaxOperandBuffer = 8ull << 30;  // per two-pass operand buffer (batches)
// Samples per tensor-core launch in a batch: long enough that the int64 accumulators (read and
// written once per launch) cost little, short enough that the operand rows the CTAs working at the
// same time share stay in L2: about kL2Window bytes of operand across the channels in flight
// (one CTA per SM / tiles per channel). Measured at 512 inputs (1 KiB of operand per sample and
// channel, 20 tiles per channel), per launch: 8192 samples 198, 16384 207, 32768 212, 49152 190,
// 65536 151 Tera-CMAC/s.
constexpr unsigned long long kL2Window = 256ull << 20;
// SM count assumed by host-only queries when no device is present (a GB300 has 152).
constexpr int kDefaultSmCount = 152;
// Multiprocessor count of the current device (cached per device; thread-safe), or kDefaultSmCount
// when no device is available.
int sm_count();

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------------------------
// Kernel launchers (each returns cudaSuccess or the launch error)
// ---------------------------------------------------------------------------------------------
cudaError_t launch_fp32(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const int2* d_tiles,
                        int n_tiles, long long* d_cross, long long* d_autos, cudaStream_t st);

// Autos (+ offset sums when d_soff != nullptr).
cudaError_t launch_autos(const Shape& s, const uint8_t* d_in, int T_blk, long long* d_autos, long long* d_soff,
                         cudaStream_t st);

// Fused unpack + tcgen05 X-engine (offset-domain products into d_cross, diagonal into d_autos).
cudaError_t launch_i8mma(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const int2* d_tiles,
                         int n_tiles, long long* d_cross, long long* d_autos, cudaStream_t st);
cudaError_t launch_f8_fused(const Shape& s, const uint8_t* d_in, int T_blk, int flush_len, const F8Tile* d_tiles,
                            int n_tiles, long long* d_cross, long long* d_autos, int* d_err, int num_sms,
                            cudaStream_t st);

// Operand build (d_op may be null) + per-input offset sums added to d_s1 and d_s2 (either may be
// null). T_blk valid samples; T_run = round_up(T_blk, kF8Kt) samples written; T_stride = op samples
// per channel.
// The block is written at sample offset t_base of each channel's operand rows.
cudaError_t launch_f8_prep(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int T_stride, int t_base, int R,
                           uint8_t* d_op, long long* d_s1, long long* d_s2, cudaStream_t st);
// The builds of several arrays (a group of sub-arrays: one block of T_blk samples each, T_run written)
// in one launch; each job as launch_f8_prep would build it alone.
struct PrepJobDesc {
  Shape s;
  const uint8_t* in;
  int T_stride, t_base, R;
  uint8_t* op;
  long long* s1;
  long long* s2;
};
cudaError_t launch_f8_prep_group(const PrepJobDesc* jobs, int n, int T_blk, int T_run, cudaStream_t st);

// The same operand bytes and offset sums built with TMA loads and stores by at most max_ctas persistent
// CTAs (one per SM), for running beside the X-engine (prep_tma.cu); f8_prep_tma_supported says whether
// the shape and buffer allow it (N % 16 == 0, N >= 128, T_blk >= 128, 16-byte aligned input).
// beside_xeng: the small variant (about 30 KB of shared memory) that fits next to an X-engine CTA on
// every SM; otherwise the wide variant for a few SMs of its own.
cudaError_t launch_f8_prep_tma(const Shape& s, const uint8_t* d_in, int T_blk, int T_run, int t_base, uint8_t* d_op,
                               long long T_span, int R_buf, long long* d_s1, long long* d_s2, int* d_err,
                               int max_ctas, bool beside_xeng, cudaStream_t st);
bool f8_prep_tma_supported(const Shape& s, const void* d_in, int T_blk);

// Offset-domain products of every work item into its array's cross sums, diagonal into its autos.
cudaError_t launch_f8_xeng(const XengArgs& args, int num_sms, cudaStream_t st);

// Tile plans of the triangle (a >= c) for N inputs with R operand rows: plan 0 = a-side spans of
// 128 inputs (N = 256 rows) with a half-width first span on odd c-blocks; plan 1 = spans of 64
// inputs (N = 128) everywhere; plan 2 = pairs of c-blocks (c0, c0 + 64) against a-spans of 128
// inputs, both halves sharing the B operand (wide mode of the two-pass X-engine): nb = half 0's
// width, pad = half 1's width | (1 << 16 when half 1 starts at the second B atom, on a diagonal
// pair); half 1's width is 0 when c0 + 64 >= N.
std::vector<F8Tile> f8_tile_plan(int N, int R, int plan);
// Tile plan 3 on pairs of SMs (xeng_pair.cu): called by launch_f8_xeng for XengArgs::pair.
cudaError_t launch_f8_xeng_pair(const XengArgs& args, int num_sms, cudaStream_t st);

size_t f8_smem_bytes();

// One-thread kernel whose bounded wait on a never-completed barrier gives up after limit_ms and
// records `code` in d_err (failure-detection self-test).
cudaError_t launch_wait_selftest(int* d_err, int limit_ms, int code, cudaStream_t st);

// Dump elements [k_base, k_base + n_elems) of an accumulator, corrected with g (cross dumps: k_base
// and n_elems even, i.e. whole (re, im) cells).
// Selective dump of the cells among stations st[0..n_st) for channels [f0, f0 + nf) (output indexed from
// channel f0); with reset, each dumped cell is set so that its corrected value restarts from zero.
cudaError_t launch_dump_select(long long* d_acc, const int* d_st, int n_st, int f0, int nf, void* d_out, int fmt,
                               long long n_samples, int reset, const Shape2& g, cudaStream_t st);
// base[b] (cross: station pairs among st) or base[i] (autos: inputs of st) = value.
cudaError_t launch_set_base(long long* d_base, const int* d_st, int n_st, long long value, const Shape2& g,
                            cudaStream_t st);
// F-engine tail: gain, round, clip to 4+4 bits, channel selection and corner turn (requant.cu).
cudaError_t launch_requant(const void* d_in, int in_type, int N, int T, int F, int chan0, int C, float gain,
                           const float* d_gains, int symmetric, uint8_t* d_out, cudaStream_t st);
// PFB F-engine: int8 ADC frames -> FIR (exact int32) -> 8192-point real FFT -> float2 [N][T][4096] (pfb.cu).
cudaError_t launch_pfb(const int8_t* d_adc, long long stride, int N, int T, int P, const int* d_h, float2* d_out,
                       cudaStream_t st);
// Unique id of the CUDA context current to this thread (binding the device's primary context if none
// is), or 0 if it cannot be read.
unsigned long long context_id();
// Raise a kernel's dynamic shared-memory limit to `bytes` in the current context, once per (kernel,
// context); thread-safe.
cudaError_t set_smem_limit(const void* func, int bytes);
cudaError_t launch_dump(const long long* d_acc, long long n_elems, void* d_out, int fmt, long long n_samples,
                        long long k_base, const Shape2& g, cudaStream_t st);

// Thread-local message returned by corr_last_error().
void set_last_error(const std::string& msg);

// Tensor-map encoding through the driver entry point (no libcuda link dependency).
// cgroup 2 or 4: boxes of R = 128 / cgroup rows x 128 samples x cgroup channels (channel groups).
int encode_op_tensor_map(CUtensorMap* map, void* d_op, int R, int T_pad, int C, std::string* err, int cgroup = 0);
// Raw input in[T][C][N] as a 3-D map, boxes of 64 inputs x 1 channel x 128 samples, no swizzle.
int encode_input_tensor_map(CUtensorMap* map, const void* d_in, int N, int C, int T, std::string* err);

// The fused path needs 16-byte TMA strides (N % 16 == 0, aligned input) and boxes no larger than the
// array (N >= 64, T >= 128).
bool f8_fused_supported(const Shape& s, const void* d_in, int T_blk);

}  // namespace corr
