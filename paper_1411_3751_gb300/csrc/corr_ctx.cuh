// Internal to libcorr (host side): the context object behind the opaque corr_ctx of include/corr.h
// and the helpers that its translation units share. Not installed, not part of the C ABI.
#pragma once

#include <string>
#include <vector>

#include "corr_internal.cuh"

namespace corr {
namespace host {

struct Layout {
  Shape s;
  long long cross_elems;  // int64 elements
  long long autos_elems;
  int R;                  // FP8 operand rows per sample as the tiles see them: round_up(2N, 128)
  int R_buf;              // operand rows stored per sample: round_up(2N, 32); the TMA fills rows
                          // R_buf .. R - 1 of a tile with zeros (out of the tensor map's extent)
  int T_pad;              // FP8 operand samples per channel and block
  size_t op_bytes;        // one block's operand
  int K_batch;            // blocks per operand buffer (one tensor-core launch in a batch)
  size_t op_buf_bytes;    // K_batch blocks' operand
  bool ok;
};

// Opt-in per-kernel timing: CUDA events recorded on the launching stream around each launch.
struct KernelTimer {
  std::vector<cudaEvent_t> ev;  // pairs (start, stop)
  size_t used = 0;
  long long launches = 0;
  double ms = 0.0;
};

}  // namespace host
}  // namespace corr

struct corr_ctx {
  corr::host::Layout L;
  bool profiling;
  corr::host::KernelTimer timers[CORR_KERNEL_COUNT];
  int path;
  int flush_len;  // 0 = path default
  int device;
  int num_sms;
  long long* d_cross;
  long long* d_autos;
  long long* d_soff;       // [C][N][2] offset sums of the tensor paths (cross cadence)
  long long* d_soff_auto;  // same, total-power cadence
  long long n_off;         // samples accumulated through a tensor path since the cross reset
  long long n_off_auto;    // same, since the autos reset
  int* d_err;
  uint8_t* d_op;          // operand scratch of the two-pass tensor path (K_batch blocks)
  CUtensorMap tmap;
  CUtensorMap tmap_cp;    // the same buffer as channel-group boxes (64 or 32 operand rows: at most 32 inputs)
  // overlapped batches: the operand of chunk j + 1 is built on prep_sms SMs (TMA build kernel, on
  // prep_stream) while the X-engine multiplies chunk j on the others; d_op2 is the second buffer
  int prep_sms;           // -1: automatic, 0: no overlap
  int K_default;          // blocks per batch launch chosen by the L2 rule (corr_set_batch_blocks 0)
  uint8_t* d_op2;
  CUtensorMap tmap2;
  CUtensorMap tmap2_cp;
  cudaStream_t prep_stream;
  cudaEvent_t ev_op_ready[2], ev_op_free[2], ev_batch_start;
  int2* d_tiles32;
  int n_tiles32;
  corr::F8Tile* d_tiles8;        // tile list (current plan), used by the fused path
  int n_tiles8;
  corr::WorkItem* d_items;       // channel-major work list of the two-pass tensor path
  long long n_items;
  int tile_plan;
  int plan_default;              // default_tile_plan(N): the plan a new context starts with
  void* d_stage[2];      // host dumps
  void* d_in_stage[2];   // host inputs
  size_t in_stage;
  cudaStream_t copy_stream;
  cudaEvent_t ev_copied[2], ev_free[2];
  bool free_recorded[2];
  int next_in;
  long long n_cross;
  long long n_auto;
  // selective dumps: station list scratch and the per-cell sample counts at the last selective reset
  int* d_sel;
  int sel_cap;
  long long* d_cross_base;  // [B_s], allocated at the first selective cross reset
  long long* d_auto_base;   // [N], allocated at the first selective autos reset
};

namespace corr {
namespace host {

// corr_last_error's message for this thread; returns code
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
// in-chip partial-sum length of `path` for this context (its setting, else the path default)
int flush_for(const corr_ctx* c, int path);
// opt-in kernel timing around a launch on st (no-ops unless profiling is on)
bool timer_begin(corr_ctx* c, int k, cudaStream_t st);
void timer_end(corr_ctx* c, int k, cudaStream_t st, bool begun);
// tile list and channel-major work list of the tensor paths for plan 0, 1 or 2
int set_tile_plan(corr_ctx* c, int plan);
// Tile plan a context of N inputs starts with: 3 (SM pairs) from 512 inputs, else 0.
int default_tile_plan(int N);
// Channels per item of an array's channel groups: 2 for 64 operand rows per channel (17 .. 32 inputs),
// 4 for 32 rows (at most 16 inputs), else 0.
int channel_group(const Layout& L);
// The two-pass X-engine of this context takes channel-group items: channel_group(L) > 0 and a one-SM
// tile plan (0 or 1).
bool uses_channel_groups(const corr_ctx* c);
// blocks per tensor-core launch of batches (reallocates the operand buffers once the device is idle)
int set_batch_blocks(corr_ctx* c, int K);
// largest blocks per launch the operand buffer cap allows for this shape
int max_batch_blocks(const corr_ctx* c);
// n device blocks through the two-pass tensor path (batch schedule of the context's settings)
int accumulate_batch_chunks(corr_ctx* c, const uint8_t* const* blocks, int n, cudaStream_t st);
// T_blk samples of a device block [T_blk][C][N] through the context's current path
int accumulate_device(corr_ctx* c, const uint8_t* d_in, int T_blk, cudaStream_t st);

}  // namespace host
}  // namespace corr
