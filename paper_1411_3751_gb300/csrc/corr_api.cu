// C ABI of libcorr: argument validation, context and memory ownership, path dispatch, dumps.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "corr_ctx.cuh"
#include "corr_internal.cuh"

#include <cmath>

using namespace corr;
using namespace corr::host;

namespace corr {
namespace host {

thread_local std::string g_err;


int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(CORR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}


constexpr size_t kStageBytes = 64ull << 20;     // host-dump staging buffer, x2
constexpr size_t kMaxInStage = 512ull << 20;    // host-input staging buffer (per buffer), x2


bool mul_ok(unsigned long long a, unsigned long long b, unsigned long long* out) {
  if (a != 0 && b > ~0ull / a) return false;
  *out = a * b;
  return true;
}

Layout make_layout(int N, int C, int T, int npol) {
  Layout L{};
  L.ok = false;
  if (N < 1 || C < 1 || T < 1 || (npol != 1 && npol != 2) || N % npol != 0) return L;
  if (N > (1 << 20) || C > 65535) return L;  // channels index grid.y of the per-channel kernels
  L.s.N = N;
  L.s.C = C;
  L.s.T = T;
  L.s.npol = npol;
  L.s.S = N / npol;
  L.s.Bs = (long long)L.s.S * (L.s.S + 1) / 2;
  L.s.P = npol * npol;
  if (L.s.Bs * L.s.P >= (1LL << 31)) return L;  // cells per channel are indexed with 32-bit integers
  unsigned long long x;
  if (!mul_ok((unsigned long long)C, (unsigned long long)L.s.Bs * L.s.P * 2, &x) || x > (1ull << 58)) return L;
  L.cross_elems = (long long)x;
  L.autos_elems = (long long)C * N;
  L.R = (int)round_up(2LL * N, kF8RowAlign);
  L.R_buf = (int)round_up(2LL * N, 32);
  L.T_pad = (int)round_up(T, kF8Kt);
  unsigned long long ob;
  if (!mul_ok((unsigned long long)C * (unsigned long long)L.T_pad, (unsigned long long)L.R_buf, &ob) || ob > (1ull << 46))
    return L;
  L.op_bytes = ob;
  // blocks per batch launch: the operand of the channels in flight within kL2Window (see there),
  // at most kF8MaxFlush samples per launch, and a buffer is capped at kMaxOperandBuffer
  const long long tiles_per_chan = (long long)f8_tile_plan(N, L.R, 0).size();
  double in_flight = (double)sm_count() / (double)(tiles_per_chan > 0 ? tiles_per_chan : 1);
  if (in_flight < 1.0) in_flight = 1.0;
  const double t_launch = (double)kL2Window / (in_flight * (double)L.R_buf);
  long long k = (long long)(t_launch / (double)L.T_pad);
  if (k * L.T_pad > kF8MaxFlush) k = kF8MaxFlush / L.T_pad;
  if (k < 1) k = 1;
  const long long kmem = ob > 0 ? (long long)(kMaxOperandBuffer / ob) : 1;
  if (k > kmem) k = kmem < 1 ? 1 : kmem;
  L.K_batch = (int)k;
  L.op_buf_bytes = ob * (size_t)k;
  L.ok = true;
  return L;
}

size_t in_stage_bytes(const Layout& L) {
  const size_t block = (size_t)L.s.T * L.s.C * L.s.N;
  return block < kMaxInStage ? block : kMaxInStage;
}

size_t footprint(const Layout& L, int path) {
  size_t b = (size_t)(L.cross_elems + L.autos_elems) * 8 + (size_t)L.autos_elems * 32 + 256;
  b += 2 * kStageBytes + 2 * in_stage_bytes(L);
  if (path == CORR_PATH_FP8TC || path == CORR_PATH_AUTO || path == CORR_PATH_FP8TC_FUSED)
    b += L.op_buf_bytes;  // operand scratch (the fused path falls back to two passes for some shapes)
  const long long nb = (L.s.N + 63) / 64;
  b += (size_t)(nb * (nb + 1) / 2) * sizeof(int2) + (size_t)(nb * 8 + 8) * sizeof(F8Tile);
  return b;
}

std::vector<int2> fp32_tiles(int N) {
  std::vector<int2> t;
  const int nb = (N + 63) / 64;
  for (int ib = 0; ib < nb; ++ib)
    for (int jb = 0; jb <= ib; ++jb) t.push_back(make_int2(ib, jb));
  return t;
}

}  // namespace host
}  // namespace corr

namespace corr {
void set_last_error(const std::string& msg) { g_err = msg; }

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return kDefaultSmCount;
  }
  static std::mutex m;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> lock(m);
  const auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = kDefaultSmCount;
  }
  cache[dev] = n;
  return n;
}

namespace {
typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);
std::once_flag g_ctx_fns_once;
ctx_get_current_fn g_ctx_get_current = nullptr;
ctx_get_id_fn g_ctx_get_id = nullptr;
}  // namespace

unsigned long long context_id() {
  std::call_once(g_ctx_fns_once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<ctx_get_current_fn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<ctx_get_id_fn>(p);
    cudaGetLastError();
  });
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) {
    // no context is current: bind the current device's primary context (cudaSetDevice creates it)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  }
  unsigned long long id = 0;
  return g_ctx_get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

cudaError_t set_smem_limit(const void* func, int bytes) {
  static std::mutex m;
  static std::set<std::pair<const void*, unsigned long long>> done;  // (kernel, context); the attribute is per context
  const unsigned long long ctx = context_id();
  std::lock_guard<std::mutex> lock(m);
  if (ctx != 0 && done.count({func, ctx})) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && ctx != 0) done.insert({func, ctx});
  return e;
}
}  // namespace corr



namespace corr {
namespace host {

int resolved_path(const corr_ctx* c) { return c->path == CORR_PATH_AUTO ? CORR_PATH_FP8TC : c->path; }

bool valid_path(int path) {
  return path == CORR_PATH_AUTO || path == CORR_PATH_FP32 || path == CORR_PATH_I8MMA || path == CORR_PATH_FP8TC ||
         path == CORR_PATH_FP8TC_FUSED;
}


int flush_for(const corr_ctx* c, int path) {
  if (c->flush_len > 0) {
    const int g = path == CORR_PATH_FP32 ? kF32Kt : kF8Kt;
    return (c->flush_len / g) * g;
  }
  return path == CORR_PATH_FP32 ? kDefaultFlushF32 : kDefaultFlushF8;
}


// Sum and recycle recorded event pairs (synchronizes on the last recorded stop event).
void drain_timer(KernelTimer& t) {
  for (size_t k = 0; k < t.used; ++k) {
    float ms = 0.f;
    if (cudaEventSynchronize(t.ev[2 * k + 1]) == cudaSuccess && cudaEventElapsedTime(&ms, t.ev[2 * k], t.ev[2 * k + 1]) == cudaSuccess)
      t.ms += ms;
  }
  t.used = 0;
}


bool timer_begin(corr_ctx* c, int k, cudaStream_t st) {
  if (!c->profiling) return false;
  KernelTimer& t = c->timers[k];
  if (t.used >= 4096) drain_timer(t);
  while (t.ev.size() < 2 * (t.used + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    t.ev.push_back(e);
  }
  cudaEventRecord(t.ev[2 * t.used], st);
  return true;
}
void timer_end(corr_ctx* c, int k, cudaStream_t st, bool begun) {
  if (!begun) return;
  KernelTimer& t = c->timers[k];
  cudaEventRecord(t.ev[2 * t.used + 1], st);
  ++t.used;
  ++t.launches;
}


void free_ctx(corr_ctx* c) {
  if (!c) return;
  for (int k = 0; k < CORR_KERNEL_COUNT; ++k)
    for (cudaEvent_t e : c->timers[k].ev) cudaEventDestroy(e);
  cudaFree(c->d_cross);
  cudaFree(c->d_autos);
  cudaFree(c->d_soff);
  cudaFree(c->d_soff_auto);
  cudaFree(c->d_err);
  cudaFree(c->d_op);
  cudaFree(c->d_tiles32);
  cudaFree(c->d_tiles8);
  cudaFree(c->d_items);
  cudaFree(c->d_stage[0]);
  cudaFree(c->d_stage[1]);
  cudaFree(c->d_in_stage[0]);
  cudaFree(c->d_in_stage[1]);
  cudaFree(c->d_sel);
  cudaFree(c->d_cross_base);
  cudaFree(c->d_auto_base);
  for (int k = 0; k < 2; ++k) {
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    if (c->ev_free[k]) cudaEventDestroy(c->ev_free[k]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  cudaFree(c->d_op2);
  for (int k = 0; k < 2; ++k) {
    if (c->ev_op_ready[k]) cudaEventDestroy(c->ev_op_ready[k]);
    if (c->ev_op_free[k]) cudaEventDestroy(c->ev_op_free[k]);
  }
  if (c->ev_batch_start) cudaEventDestroy(c->ev_batch_start);
  if (c->prep_stream) cudaStreamDestroy(c->prep_stream);
  delete c;
}

XengArgs xeng_args(const corr_ctx* c, int buf, int T_run, int flush);  // buf: operand buffer d_op (0) or d_op2 (1)

// Accumulate T_blk samples from a device buffer laid out [T_blk][C][N].

int accumulate_device(corr_ctx* c, const uint8_t* d_in, int T_blk, cudaStream_t st) {
  const int path = resolved_path(c);
  const int flush = flush_for(c, path);
  cudaError_t e;
  if (path == CORR_PATH_FP32) {
    const bool tb = timer_begin(c, CORR_KERNEL_XENG, st);
    e = launch_fp32(c->L.s, d_in, T_blk, flush, c->d_tiles32, c->n_tiles32, c->d_cross, c->d_autos, st);
    timer_end(c, CORR_KERNEL_XENG, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "fp32 x-engine launch");
  } else if (path == CORR_PATH_I8MMA) {
    const bool tb = timer_begin(c, CORR_KERNEL_XENG, st);
    e = launch_i8mma(c->L.s, d_in, T_blk, flush, c->d_tiles32, c->n_tiles32, c->d_cross, c->d_autos, st);
    timer_end(c, CORR_KERNEL_XENG, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "int8 mma x-engine launch");
  } else {
    // tensor paths: one pass builds the operand (two-pass path) and the per-input offset sums for
    // both cadences; the X-engine adds the offset-domain products and their diagonal.
    const int T_run = (int)round_up(T_blk, kF8Kt);
    const bool two_pass = path == CORR_PATH_FP8TC || !f8_fused_supported(c->L.s, d_in, T_blk);
    bool tb = timer_begin(c, CORR_KERNEL_UNPACK, st);
    e = launch_f8_prep(c->L.s, d_in, T_blk, T_run, c->L.T_pad * c->L.K_batch, 0, c->L.R_buf, two_pass ? c->d_op : nullptr,
                       c->d_soff,
                       c->d_soff_auto, st);
    timer_end(c, CORR_KERNEL_UNPACK, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "operand build launch");
    tb = timer_begin(c, CORR_KERNEL_XENG, st);
    if (two_pass)
      e = launch_f8_xeng(xeng_args(c, 0, T_run, flush), c->num_sms, st);
    else
      e = launch_f8_fused(c->L.s, d_in, T_blk, flush, c->d_tiles8, c->n_tiles8, c->d_cross, c->d_autos, c->d_err,
                          c->num_sms, st);
    timer_end(c, CORR_KERNEL_XENG, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "tensor x-engine launch");
    c->n_off += T_blk;
    c->n_off_auto += T_blk;
  }
  return CORR_OK;
}


// Tile plan of the tensor paths: the tile list (fused path) and the channel-major work list
// (two-pass path) for plan 0, 1 or 2 (see f8_tile_plan).

int set_tile_plan(corr_ctx* c, int plan) {
  // the fused path has no wide mode: it keeps plan 0 under plan 2
  const std::vector<F8Tile> t8 = f8_tile_plan(c->L.s.N, c->L.R, plan >= 2 ? 0 : plan);
  const std::vector<F8Tile> tw = plan >= 2 ? f8_tile_plan(c->L.s.N, c->L.R, plan) : t8;
  std::vector<WorkItem> items;
  items.reserve((size_t)c->L.s.C * tw.size());
  if (channel_group(c->L) > 0 && plan < 2) {  // channel groups (uses_channel_groups)
    for (int f = 0; f < c->L.s.C; f += channel_group(c->L)) items.push_back(WorkItem{0, f, 0, 0, 128, 0});
  } else {
    for (int f = 0; f < c->L.s.C; ++f)
      for (const F8Tile& t : tw) items.push_back(WorkItem{0, f, t.c0, t.a0, t.nb, t.pad});
  }
  F8Tile* d_t = nullptr;
  WorkItem* d_i = nullptr;
  if (cudaMalloc(&d_t, t8.size() * sizeof(F8Tile)) != cudaSuccess ||
      cudaMalloc(&d_i, items.size() * sizeof(WorkItem)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_t);
    return fail(CORR_ERR_OOM, "tile list allocation failed");
  }
  cudaError_t e = cudaMemcpy(d_t, t8.data(), t8.size() * sizeof(F8Tile), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_i, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d_t);
    cudaFree(d_i);
    return cuda_fail(e, "tile list upload");
  }
  cudaFree(c->d_tiles8);
  cudaFree(c->d_items);
  c->d_tiles8 = d_t;
  c->n_tiles8 = (int)t8.size();
  c->d_items = d_i;
  c->n_items = (long long)items.size();
  c->tile_plan = plan;
  return CORR_OK;
}


int default_tile_plan(int N) {
  // measured at 512 inputs, 128 channels, 4 x 8192 samples per launch: plan 3 1.35-1.37 ms per launch,
  // plan 0 1.44-1.46 ms; below 512 inputs the 128-input tiles of plan 3 waste a larger share of their
  // products on the diagonal (a quarter of them at 256 inputs against a tenth at 512)
  return N >= 512 ? 3 : 0;
}

int channel_group(const Layout& L) { return L.R_buf == 64 ? 2 : (L.R_buf == 32 ? 4 : 0); }

bool uses_channel_groups(const corr_ctx* c) { return channel_group(c->L) > 0 && c->tile_plan < 2; }

XengArgs xeng_args(const corr_ctx* c, int buf, int T_run, int flush) {
  XengArgs a;
  std::memset(&a, 0, sizeof(a));
  const bool cp = uses_channel_groups(c);
  a.a[0].tmap = cp ? (buf ? c->tmap2_cp : c->tmap_cp) : (buf ? c->tmap2 : c->tmap);
  a.a[0].C = c->L.s.C;
  a.a[0].cgroup = cp ? channel_group(c->L) : 0;
  a.a[0].cross = c->d_cross;
  a.a[0].autos = c->d_autos;
  a.a[0].Bs = c->L.s.Bs;
  a.a[0].N = c->L.s.N;
  a.a[0].npol = c->L.s.npol;
  a.items = c->d_items;
  a.n_items = c->n_items;
  a.T_run = T_run;
  a.flush_len = flush;
  a.err = c->d_err;
  a.wide = c->tile_plan == 2 ? 1 : 0;
  a.pair = c->tile_plan == 3 ? 1 : 0;
  return a;
}

// The two-pass tensor path's operand scratch and its TMA tensor map.
int ensure_operand_scratch(corr_ctx* c) {
  if (c->d_op) return CORR_OK;
  if (cudaMalloc(&c->d_op, c->L.op_buf_bytes) != cudaSuccess) {
    cudaGetLastError();
    c->d_op = nullptr;
    return fail(CORR_ERR_OOM, "operand scratch allocation failed");
  }
  cudaError_t e = cudaMemset(c->d_op, 0, c->L.op_buf_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "operand scratch init");
  std::string err;
  if (encode_op_tensor_map(&c->tmap, c->d_op, c->L.R_buf, c->L.T_pad * c->L.K_batch, c->L.s.C, &err) != 0 ||
      (channel_group(c->L) > 0 && encode_op_tensor_map(&c->tmap_cp, c->d_op, c->L.R_buf, c->L.T_pad * c->L.K_batch,
                                                       c->L.s.C, &err, channel_group(c->L)) != 0)) {
    cudaFree(c->d_op);
    c->d_op = nullptr;
    return fail(CORR_ERR_CUDA, err);
  }
  return CORR_OK;
}

int max_batch_blocks(const corr_ctx* c) {
  const unsigned long long ob = c->L.op_bytes > 0 ? c->L.op_bytes : 1;
  const unsigned long long k = kMaxOperandBuffer / ob;
  return k < 1 ? 1 : (k > 64 ? 64 : (int)k);
}

int set_batch_blocks(corr_ctx* c, int K) {
  if (K == c->L.K_batch) return CORR_OK;
  const cudaError_t e = cudaDeviceSynchronize();  // queued launches read the current buffers
  if (e != cudaSuccess) return cuda_fail(e, "set_batch_blocks: synchronize");
  const bool had_op = c->d_op != nullptr;
  const int old_K = c->L.K_batch;
  cudaFree(c->d_op);
  cudaFree(c->d_op2);
  c->d_op = nullptr;
  c->d_op2 = nullptr;
  c->L.K_batch = K;
  c->L.op_buf_bytes = c->L.op_bytes * (size_t)K;
  if (!had_op) return CORR_OK;
  const int rc = ensure_operand_scratch(c);
  if (rc == CORR_OK) return CORR_OK;
  const std::string msg = g_err;
  c->L.K_batch = old_K;  // back to the old size, which fitted before
  c->L.op_buf_bytes = c->L.op_bytes * (size_t)old_K;
  ensure_operand_scratch(c);
  return fail(rc, msg);
}

// SMs that build the next chunk's operand while the X-engine multiplies the current one.
int prep_sms_for(const corr_ctx* c) {
  if (c->prep_sms >= 0) return c->prep_sms;
  // automatic: sequential; corr_autotune times the overlapped schedules on the caller's blocks.
  // Measured at 512 inputs x 128 channels x 16 blocks of 8192 samples: with the one-SM plan 0, 217.7
  // Tera-CMAC/s in sequence, 209.4 with the build on 38 SMs of its own, 187.6 with a small build CTA
  // beside the X-engine on every SM (the X-engine slows by more than the SMs it gives up); with the
  // SM-pair plan 3, 236.3 in sequence and 240.2 / 252.4 / 244.5 with the build on 38 / 42 / 46 SMs
  // (the X-engine now slows in proportion to the SMs it gives up; the best k balances a build of a
  // launch's blocks on k SMs against their multiply on the others)
  return 0;
}

// The second operand buffer (with its X-engine tensor map) and the stream and events of overlapped
// batches (allocated on first use).
int ensure_overlap(corr_ctx* c) {
  std::string err;
  if (!c->d_op2) {
    if (cudaMalloc(&c->d_op2, c->L.op_buf_bytes) != cudaSuccess) {
      cudaGetLastError();
      c->d_op2 = nullptr;
      return fail(CORR_ERR_OOM, "second operand buffer allocation failed");
    }
    cudaError_t e = cudaMemset(c->d_op2, 0, c->L.op_buf_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "second operand buffer init");
    if (encode_op_tensor_map(&c->tmap2, c->d_op2, c->L.R_buf, c->L.T_pad * c->L.K_batch, c->L.s.C, &err) != 0 ||
        (channel_group(c->L) > 0 && encode_op_tensor_map(&c->tmap2_cp, c->d_op2, c->L.R_buf,
                                                         c->L.T_pad * c->L.K_batch, c->L.s.C, &err,
                                                         channel_group(c->L)) != 0)) {
      cudaFree(c->d_op2);
      c->d_op2 = nullptr;
      return fail(CORR_ERR_CUDA, err);
    }
  }
  if (!c->prep_stream) {
    bool ok = cudaStreamCreateWithFlags(&c->prep_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
      ok = cudaEventCreateWithFlags(&c->ev_op_ready[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->ev_op_free[k], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventCreateWithFlags(&c->ev_batch_start, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_fail(cudaGetLastError(), "overlap stream / events");
  }
  return CORR_OK;
}

// n blocks in chunks of K_batch blocks, the operand build of chunk j + 1 overlapping the multiply of
// chunk j: the build (TMA loads, 16-byte stores) runs on the context's build stream into one operand
// buffer while the X-engine multiplies the other buffer on the caller's stream; events order each
// buffer's reuse. k < SMs: the build has k SMs to itself and the X-engine the others; k == SMs: a
// small build CTA shares every SM with an X-engine CTA. The first build and the last multiply have
// the GPU to themselves.
int accumulate_batch_overlap(corr_ctx* c, const uint8_t* const* blocks, int n, cudaStream_t st, int k) {
  const int T_blk = c->L.s.T;
  const int T_pad = c->L.T_pad;
  const int K = c->L.K_batch;
  const int flush = flush_for(c, CORR_PATH_FP8TC);
  const int S = c->num_sms;
  const int rc = ensure_overlap(c);
  if (rc != CORR_OK) return rc;
  cudaStream_t ps = c->prep_stream;
  cudaError_t e = cudaEventRecord(c->ev_batch_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, c->ev_batch_start, 0);
  const int J = (n + K - 1) / K;
  for (int j = 0; j < J && e == cudaSuccess; ++j) {
    const int buf = j & 1;
    const int b0 = j * K;
    const int nb = (n - b0) < K ? (n - b0) : K;
    if (j >= 2) e = cudaStreamWaitEvent(ps, c->ev_op_free[buf], 0);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
      const bool tb = timer_begin(c, CORR_KERNEL_UNPACK, ps);
      if (j == 0)  // nothing to overlap with yet: the whole-GPU build
        e = launch_f8_prep(c->L.s, blocks[b0 + i], T_blk, T_pad, T_pad * K, i * T_pad, c->L.R_buf,
                           buf ? c->d_op2 : c->d_op, c->d_soff, c->d_soff_auto, ps);
      else
        e = launch_f8_prep_tma(c->L.s, blocks[b0 + i], T_blk, T_pad, i * T_pad, buf ? c->d_op2 : c->d_op,
                               (long long)T_pad * K, c->L.R_buf, c->d_soff, c->d_soff_auto, c->d_err, k, k >= S, ps);
      timer_end(c, CORR_KERNEL_UNPACK, ps, tb);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_op_ready[buf], ps);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_op_ready[buf], 0);
    if (e == cudaSuccess) {
      const bool tb = timer_begin(c, CORR_KERNEL_XENG, st);
      // k == S: the build shares every SM with the X-engine (one small build CTA beside each X-engine CTA)
      const int grid_x = (j == J - 1 || k >= S) ? S : S - k;
      e = launch_f8_xeng(xeng_args(c, buf, nb * T_pad, flush), grid_x, st);
      timer_end(c, CORR_KERNEL_XENG, st, tb);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_op_free[buf], st);
    c->n_off += (long long)T_blk * nb;
    c->n_off_auto += (long long)T_blk * nb;
  }
  if (e != cudaSuccess) return cuda_fail(e, "overlapped batch");
  return CORR_OK;
}

// n blocks through the two-pass tensor path in chunks of up to K_batch blocks (launch length from the
// L2 budget, see kL2Window): the operand of a chunk is built with each block at its own sample
// offset, then one tensor-core launch multiplies the whole chunk, so blocks share launches and
// flushes. With prep_sms_for(c) = k > 0 the build of chunk j + 1 runs on k SMs beside the multiply of
// chunk j (accumulate_batch_overlap); otherwise the chunks run in order on the caller's stream.
int accumulate_batch_chunks(corr_ctx* c, const uint8_t* const* blocks, int n, cudaStream_t st) {
  // overlapped schedule when there are at least two chunks and the TMA build takes the shape (the wide
  // plan 2 fills both accumulators per item and is not overlapped)
  const int k = prep_sms_for(c);
  if (k > 0 && k <= c->num_sms && n > c->L.K_batch && c->tile_plan != 2) {
    bool ok = true;
    for (int b = 0; b < n && ok; ++b) ok = f8_prep_tma_supported(c->L.s, blocks[b], c->L.s.T);
    if (ok) {
      const int rc = accumulate_batch_overlap(c, blocks, n, st, k);
      if (rc != CORR_ERR_OOM) return rc;
      cudaGetLastError();  // no room for the second buffer: the sequential schedule below
    }
  }
  const int T_blk = c->L.s.T;
  const int T_pad = c->L.T_pad;
  const int K = c->L.K_batch;
  const int T_span = T_pad * K;
  const int flush = flush_for(c, CORR_PATH_FP8TC);
  for (int b0 = 0; b0 < n; b0 += K) {
    const int nb = (n - b0) < K ? (n - b0) : K;
    for (int i = 0; i < nb; ++i) {
      const bool tb = timer_begin(c, CORR_KERNEL_UNPACK, st);
      const cudaError_t e = launch_f8_prep(c->L.s, blocks[b0 + i], T_blk, T_pad, T_span, i * T_pad, c->L.R_buf, c->d_op,
                                           c->d_soff, c->d_soff_auto, st);
      timer_end(c, CORR_KERNEL_UNPACK, st, tb);
      if (e != cudaSuccess) return cuda_fail(e, "batch operand build");
    }
    const bool tb = timer_begin(c, CORR_KERNEL_XENG, st);
    const cudaError_t e = launch_f8_xeng(xeng_args(c, 0, nb * T_pad, flush), c->num_sms, st);
    timer_end(c, CORR_KERNEL_XENG, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "batch x-engine");
    c->n_off += (long long)T_blk * nb;
    c->n_off_auto += (long long)T_blk * nb;
  }
  return CORR_OK;
}

}  // namespace host
}  // namespace corr

extern "C" {

const char* corr_last_error(void) { return g_err.c_str(); }

const char* corr_version(void) { return "libcorr 0.1 (sm_103a)"; }

long long corr_n_baselines(int n_inputs, int n_pol) {
  if (n_inputs < 1 || (n_pol != 1 && n_pol != 2) || n_inputs % n_pol) return 0;
  const long long s = n_inputs / n_pol;
  return s * (s + 1) / 2;
}

int corr_batch_blocks(int n_inputs, int n_chans, int n_time_per_block, int n_pol) {
  const Layout L = make_layout(n_inputs, n_chans, n_time_per_block, n_pol);
  return L.ok ? L.K_batch : 0;
}

size_t corr_footprint_bytes(int n_inputs, int n_chans, int n_time_per_block, int n_pol, int path) {
  const Layout L = make_layout(n_inputs, n_chans, n_time_per_block, n_pol);
  if (!L.ok || !valid_path(path)) return 0;
  return footprint(L, path);
}

corr_ctx* corr_create(int n_inputs, int n_chans, int n_time_per_block, int n_pol) {
  const Layout L = make_layout(n_inputs, n_chans, n_time_per_block, n_pol);
  if (!L.ok) {
    fail(CORR_ERR_ARG, "corr_create: invalid shape (need N >= 1, B_s n_pol^2 < 2^31, 1 <= C <= 65535, T >= 1, "
                       "n_pol in {1,2}, N % n_pol == 0, sizes within range)");
    return nullptr;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cuda_fail(e, "corr_create: cudaGetDevice");
    return nullptr;
  }
  size_t free_b = 0, total_b = 0;
  e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    cuda_fail(e, "corr_create: cudaMemGetInfo");
    return nullptr;
  }
  if (footprint(L, CORR_PATH_AUTO) > free_b) {
    fail(CORR_ERR_OOM, "corr_create: footprint " + std::to_string(footprint(L, CORR_PATH_AUTO)) +
                           " bytes exceeds free device memory " + std::to_string(free_b));
    return nullptr;
  }
  corr_ctx* c = new (std::nothrow) corr_ctx{};
  if (!c) {
    fail(CORR_ERR_OOM, "corr_create: host allocation");
    return nullptr;
  }
  c->L = L;
  c->path = CORR_PATH_AUTO;
  c->prep_sms = -1;
  c->K_default = L.K_batch;
  c->device = dev;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (c->num_sms < 1) c->num_sms = 1;

  const std::vector<int2> t32 = fp32_tiles(L.s.N);
  c->n_tiles32 = (int)t32.size();
  bool ok = cudaMalloc(&c->d_cross, (size_t)L.cross_elems * 8) == cudaSuccess &&
            cudaMalloc(&c->d_autos, (size_t)L.autos_elems * 8) == cudaSuccess &&
            cudaMalloc(&c->d_soff, (size_t)L.autos_elems * 16) == cudaSuccess &&
            cudaMalloc(&c->d_soff_auto, (size_t)L.autos_elems * 16) == cudaSuccess &&
            cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&c->d_tiles32, t32.size() * sizeof(int2)) == cudaSuccess &&
            cudaMalloc(&c->d_stage[0], kStageBytes) == cudaSuccess &&
            cudaMalloc(&c->d_stage[1], kStageBytes) == cudaSuccess &&
            cudaMalloc(&c->d_in_stage[0], in_stage_bytes(L)) == cudaSuccess &&
            cudaMalloc(&c->d_in_stage[1], in_stage_bytes(L)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_copied[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_copied[1], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_free[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->ev_free[1], cudaEventDisableTiming) == cudaSuccess;
  c->in_stage = in_stage_bytes(L);
  if (!ok) {
    cudaGetLastError();
    free_ctx(c);
    fail(CORR_ERR_OOM, "corr_create: device allocation failed");
    return nullptr;
  }
  ok = cudaMemset(c->d_cross, 0, (size_t)L.cross_elems * 8) == cudaSuccess &&
       cudaMemset(c->d_autos, 0, (size_t)L.autos_elems * 8) == cudaSuccess &&
       cudaMemset(c->d_soff, 0, (size_t)L.autos_elems * 16) == cudaSuccess &&
       cudaMemset(c->d_soff_auto, 0, (size_t)L.autos_elems * 16) == cudaSuccess &&
       cudaMemset(c->d_err, 0, sizeof(int)) == cudaSuccess &&
       cudaMemcpy(c->d_tiles32, t32.data(), t32.size() * sizeof(int2), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    e = cudaGetLastError();
    free_ctx(c);
    cuda_fail(e, "corr_create: initialisation");
    return nullptr;
  }
  c->plan_default = default_tile_plan(L.s.N);
  if (set_tile_plan(c, c->plan_default) != CORR_OK || ensure_operand_scratch(c) != CORR_OK) {
    const std::string msg = g_err;
    free_ctx(c);
    fail(CORR_ERR_OOM, "corr_create: " + msg);
    return nullptr;
  }
  return c;
}

int corr_set_path(corr_ctx* c, int path) {
  if (!c) return fail(CORR_ERR_ARG, "corr_set_path: NULL context");
  if (!valid_path(path)) return fail(CORR_ERR_ARG, "corr_set_path: unknown path " + std::to_string(path));
  if (path == CORR_PATH_FP8TC || path == CORR_PATH_AUTO || path == CORR_PATH_FP8TC_FUSED) {
    const int rc = ensure_operand_scratch(c);  // the fused path falls back to two passes for some shapes
    if (rc != CORR_OK) return rc;
  } else if (c->d_op) {
    // FP32 and int8 paths unpack in shared memory: release the operand scratch once queued work is done
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "corr_set_path: synchronize");
    cudaFree(c->d_op);
    c->d_op = nullptr;
  }
  c->path = path;
  return CORR_OK;
}

int corr_get_path(const corr_ctx* c) { return c ? resolved_path(c) : CORR_ERR_ARG; }

int corr_set_tile_plan(corr_ctx* c, int plan) {
  if (!c) return fail(CORR_ERR_ARG, "corr_set_tile_plan: NULL context");
  if (plan < 0 || plan > 3) return fail(CORR_ERR_ARG, "corr_set_tile_plan: plan must be 0, 1, 2 or 3");
  // the work lists are read by queued launches: replace them once those are done
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "corr_set_tile_plan: synchronize");
  return set_tile_plan(c, plan);
}

int corr_get_tile_plan(const corr_ctx* c) { return c ? c->tile_plan : CORR_ERR_ARG; }

int corr_set_prep_sms(corr_ctx* c, int sms) {
  if (!c) return fail(CORR_ERR_ARG, "corr_set_prep_sms: NULL context");
  if (sms < -1 || sms > c->num_sms)
    return fail(CORR_ERR_ARG, "corr_set_prep_sms: need -1 (automatic), 0 (no overlap) or 1 .. SMs");
  c->prep_sms = sms;
  return CORR_OK;
}

int corr_get_prep_sms(const corr_ctx* c) { return c ? prep_sms_for(c) : CORR_ERR_ARG; }

int corr_set_batch_blocks(corr_ctx* c, int blocks) {
  if (!c) return fail(CORR_ERR_ARG, "corr_set_batch_blocks: NULL context");
  const int kmax = max_batch_blocks(c);
  if (blocks < 0 || blocks > kmax)
    return fail(CORR_ERR_ARG, "corr_set_batch_blocks: need 0 (the default) .. " + std::to_string(kmax) +
                                  " (an 8 GiB operand buffer) for this shape");
  return set_batch_blocks(c, blocks == 0 ? c->K_default : blocks);
}

int corr_get_batch_blocks(const corr_ctx* c) { return c ? c->L.K_batch : CORR_ERR_ARG; }

namespace {
std::mutex g_ctx_tune_mu;
// (N, C, T, n_pol, SMs, blocks) -> (plan, blocks per launch, build SMs, ms per block)
std::map<std::tuple<int, int, int, int, int, int>, std::tuple<int, int, int, double>> g_ctx_tune;
bool g_ctx_tune_loaded = false;

void ctx_tune_load() {
  if (g_ctx_tune_loaded) return;
  g_ctx_tune_loaded = true;
  const char* path = std::getenv("CORR_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return;
  char tag[16];
  int a, b, cc, d, e, f, p, k, q;
  double ms;
  while (std::fscanf(fh, "%15s", tag) == 1) {
    if (std::strcmp(tag, "batch") == 0 &&
        std::fscanf(fh, "%d %d %d %d %d %d %d %d %d %lf", &a, &b, &cc, &d, &e, &f, &p, &k, &q, &ms) == 10)
      g_ctx_tune[std::make_tuple(a, b, cc, d, e, f)] = std::make_tuple(p, k, q, ms);
    else {
      int ch;  // skip the rest of a line of another kind
      while ((ch = std::fgetc(fh)) != EOF && ch != '\n') {
      }
    }
  }
  std::fclose(fh);
}

void ctx_tune_store(const std::tuple<int, int, int, int, int, int>& key, const std::tuple<int, int, int, double>& v) {
  g_ctx_tune[key] = v;
  const char* path = std::getenv("CORR_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "batch %d %d %d %d %d %d %d %d %d %.6f\n", std::get<0>(key), std::get<1>(key), std::get<2>(key),
               std::get<3>(key), std::get<4>(key), std::get<5>(key), std::get<0>(v), std::get<1>(v), std::get<2>(v),
               std::get<3>(v));
  std::fclose(fh);
}
}  // namespace

int corr_autotune(corr_ctx* c, const void* const* d_blocks, int n_blocks, int reps, corr_tuning* out, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_autotune: NULL context");
  if (n_blocks < 1 || !d_blocks || reps < 1 || reps > 100)
    return fail(CORR_ERR_ARG, "corr_autotune: need n_blocks >= 1 blocks and 1 <= reps <= 100");
  for (int b = 0; b < n_blocks; ++b)
    if (!d_blocks[b]) return fail(CORR_ERR_ARG, "corr_autotune: NULL block " + std::to_string(b));
  if (resolved_path(c) != CORR_PATH_FP8TC)
    return fail(CORR_ERR_STATE, "corr_autotune: tunes the two-pass tensor path (CORR_PATH_FP8TC / AUTO)");
  cudaStream_t st = (cudaStream_t)stream;
  const uint8_t* const* blocks = reinterpret_cast<const uint8_t* const*>(d_blocks);
  std::lock_guard<std::mutex> lock(g_ctx_tune_mu);
  ctx_tune_load();
  const auto key = std::make_tuple(c->L.s.N, c->L.s.C, c->L.s.T, c->L.s.npol, c->num_sms, n_blocks);
  int best_plan = c->tile_plan, best_K = c->L.K_batch, best_prep = prep_sms_for(c), tried = 0;
  double best_ms = 0.0;
  int rc = CORR_OK;
  const auto hit = g_ctx_tune.find(key);
  if (hit != g_ctx_tune.end()) {
    std::tie(best_plan, best_K, best_prep, best_ms) = hit->second;
  } else {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "corr_autotune: events");
    bool tma_ok = true;
    for (int b = 0; b < n_blocks; ++b) tma_ok = tma_ok && f8_prep_tma_supported(c->L.s, blocks[b], c->L.s.T);
    // candidates: the default schedule (the shape's default plan and launch length, sequential) first;
    // another replaces the best so far only when it is at least 1% faster, so near-ties keep the default
    std::vector<std::tuple<int, int, int>> cand;
    cand.emplace_back(c->plan_default, c->K_default, 0);
    std::vector<int> Ks = {1, 2, 4, 8, c->K_default};
    std::sort(Ks.begin(), Ks.end());
    Ks.erase(std::unique(Ks.begin(), Ks.end()), Ks.end());
    for (int plan = 0; plan <= 3; ++plan)
      for (int K : Ks) {
        if (K > max_batch_blocks(c) || (K > n_blocks && K != c->K_default)) continue;
        // concurrent build SMs: fractions of the GPU around the balance of a build of K blocks on k
        // SMs against a multiply of K blocks on the others (about 2/7 at 512 inputs on plan 3), and
        // for the one-SM plans a small build CTA beside the X-engine on every SM (which the 224 KB
        // ring of a plan-3 CTA leaves no room for)
        std::vector<int> preps = {0};
        if (tma_ok && plan != 2 && n_blocks > K) {
          const int S = c->num_sms;
          for (int k : {S / 5, S / 4, 2 * S / 7, S / 3}) preps.push_back(k);
          if (plan < 2) preps.push_back(S);
        }
        for (int prep : preps)
          if (!(plan == c->plan_default && K == c->K_default && prep == 0)) cand.emplace_back(plan, K, prep);
      }
    best_ms = 1e300;
    for (const auto& cd : cand) {
      if (rc != CORR_OK) break;
      const int plan = std::get<0>(cd), K = std::get<1>(cd), prep = std::get<2>(cd);
      if (c->tile_plan != plan && (rc = set_tile_plan(c, plan)) != CORR_OK) break;
      if ((rc = set_batch_blocks(c, K)) != CORR_OK) {
        if (rc != CORR_ERR_OOM) break;
        rc = CORR_OK;  // this launch length does not fit: skip it
        continue;
      }
      c->prep_sms = prep;
      float ms = 0.f;
      for (int rep = 0; rep <= reps && rc == CORR_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        rc = accumulate_batch_chunks(c, blocks, n_blocks, st);
      }
      if (rc != CORR_OK) break;
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "corr_autotune: timing");
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      const double per_block = (double)ms / reps / n_blocks;
      ++tried;
      if (per_block < 0.99 * best_ms) {
        best_ms = per_block;
        best_plan = plan;
        best_K = K;
        best_prep = prep;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == CORR_OK) ctx_tune_store(key, std::make_tuple(best_plan, best_K, best_prep, best_ms));
  }
  if (rc == CORR_OK) rc = set_tile_plan(c, best_plan);
  if (rc == CORR_OK) rc = set_batch_blocks(c, best_K);
  c->prep_sms = best_prep;
  // the trials added into the accumulators: start from zero
  if (rc == CORR_OK) rc = corr_reset(c, CORR_WHAT_CROSS | CORR_WHAT_AUTO, stream);
  if (rc == CORR_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "corr_autotune: synchronize");
  }
  if (rc != CORR_OK) return rc;
  if (out) {
    out->tile_plan = best_plan;
    out->batch_blocks = best_K;
    out->prep_sms = best_prep;
    out->n_tried = tried;
    out->ms_per_block = best_ms;
  }
  return CORR_OK;
}

int corr_tile_plan(int n_inputs, int plan, int* tiles_out, int max_tiles) {
  if (n_inputs < 1 || n_inputs > (1 << 20) || plan < 0 || plan > 3 || max_tiles < 0 || (max_tiles > 0 && !tiles_out))
    return fail(CORR_ERR_ARG, "corr_tile_plan: need 1 <= n_inputs <= 2^20, plan 0..3, a buffer for max_tiles > 0");
  const int R = (int)round_up(2LL * n_inputs, kF8RowAlign);
  const std::vector<F8Tile> t = f8_tile_plan(n_inputs, R, plan);
  if (t.size() > (size_t)0x7fffffff) return fail(CORR_ERR_ARG, "corr_tile_plan: too many tiles");
  const int n = (int)t.size() < max_tiles ? (int)t.size() : max_tiles;
  for (int i = 0; i < n; ++i) {
    tiles_out[4 * i] = t[i].c0;
    tiles_out[4 * i + 1] = t[i].a0;
    tiles_out[4 * i + 2] = t[i].nb;
    tiles_out[4 * i + 3] = t[i].pad;
  }
  return (int)t.size();
}

int corr_channel_group(int n_inputs, int plan) {
  if (n_inputs < 1 || n_inputs > (1 << 20) || plan < 0 || plan > 3)
    return fail(CORR_ERR_ARG, "corr_channel_group: need 1 <= n_inputs <= 2^20, plan 0..3");
  Layout L{};
  L.R_buf = (int)round_up(2LL * n_inputs, 32);
  const int g = plan < 2 ? channel_group(L) : 0;
  return g > 1 ? g : 1;
}

int corr_selftest_wait(corr_ctx* c, int limit_ms, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_selftest_wait: NULL context");
  if (limit_ms < 1 || limit_ms > 2000) return fail(CORR_ERR_ARG, "corr_selftest_wait: limit_ms must be in [1, 2000]");
  const cudaError_t e = launch_wait_selftest(c->d_err, limit_ms, 90, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "corr_selftest_wait: launch");
  return CORR_OK;
}

int corr_set_flush_period(corr_ctx* c, int n) {
  if (!c) return fail(CORR_ERR_ARG, "corr_set_flush_period: NULL context");
  if (n < 0 || n > kF8MaxFlush) return fail(CORR_ERR_ARG, "corr_set_flush_period: must be in [0, 65536]");
  const int g = resolved_path(c) == CORR_PATH_FP32 ? kF32Kt : kF8Kt;
  if (n > 0 && n < g)
    return fail(CORR_ERR_ARG, "corr_set_flush_period: below the path granule " + std::to_string(g));
  c->flush_len = n;
  return CORR_OK;
}

int corr_accumulate(corr_ctx* c, const void* d_samples, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_accumulate: NULL context");
  if (!d_samples) return fail(CORR_ERR_ARG, "corr_accumulate: NULL samples");
  const int rc = accumulate_device(c, static_cast<const uint8_t*>(d_samples), c->L.s.T, (cudaStream_t)stream);
  if (rc != CORR_OK) return rc;
  c->n_cross += c->L.s.T;
  c->n_auto += c->L.s.T;
  return CORR_OK;
}

int corr_accumulate_batch(corr_ctx* c, const void* const* d_blocks, int n_blocks, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_accumulate_batch: NULL context");
  if (n_blocks < 0 || (n_blocks > 0 && !d_blocks)) return fail(CORR_ERR_ARG, "corr_accumulate_batch: bad block list");
  for (int b = 0; b < n_blocks; ++b)
    if (!d_blocks[b]) return fail(CORR_ERR_ARG, "corr_accumulate_batch: NULL block " + std::to_string(b));
  cudaStream_t st = (cudaStream_t)stream;
  const uint8_t* const* blocks = reinterpret_cast<const uint8_t* const*>(d_blocks);
  int rc = CORR_OK;
  if (resolved_path(c) == CORR_PATH_FP8TC && n_blocks > 1) {
    rc = accumulate_batch_chunks(c, blocks, n_blocks, st);
  } else {
    for (int b = 0; b < n_blocks && rc == CORR_OK; ++b) rc = accumulate_device(c, blocks[b], c->L.s.T, st);
  }
  if (rc != CORR_OK) return rc;
  c->n_cross += (long long)c->L.s.T * n_blocks;
  c->n_auto += (long long)c->L.s.T * n_blocks;
  return CORR_OK;
}

int corr_accumulate_host(corr_ctx* c, const void* h_samples, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_accumulate_host: NULL context");
  if (!h_samples) return fail(CORR_ERR_ARG, "corr_accumulate_host: NULL samples");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t row = (size_t)c->L.s.C * c->L.s.N;  // bytes per time sample
  long long slice = (long long)(c->in_stage / row);
  if (slice >= c->L.s.T) slice = c->L.s.T;
  else if (slice >= kF8Kt) slice = slice / kF8Kt * kF8Kt;
  if (slice < 1) return fail(CORR_ERR_ARG, "corr_accumulate_host: one time sample exceeds the staging buffer");
  const uint8_t* src = static_cast<const uint8_t*>(h_samples);
  // Double-buffered: the copy stream fills staging buffer k while the caller's stream computes on
  // the other; events order reuse of a buffer after the kernels that read it.
  for (long long t0 = 0; t0 < c->L.s.T; t0 += slice) {
    const int n = (int)((c->L.s.T - t0) < slice ? (c->L.s.T - t0) : slice);
    const int buf = c->next_in;
    c->next_in ^= 1;
    cudaError_t e = cudaSuccess;
    if (c->free_recorded[buf]) e = cudaStreamWaitEvent(c->copy_stream, c->ev_free[buf], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->d_in_stage[buf], src + (size_t)t0 * row, (size_t)n * row, cudaMemcpyHostToDevice,
                          c->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_copied[buf], c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_copied[buf], 0);
    if (e != cudaSuccess) return cuda_fail(e, "corr_accumulate_host: copy");
    const int rc = accumulate_device(c, static_cast<const uint8_t*>(c->d_in_stage[buf]), n, st);
    if (rc != CORR_OK) return rc;
    e = cudaEventRecord(c->ev_free[buf], st);
    if (e != cudaSuccess) return cuda_fail(e, "corr_accumulate_host: event");
    c->free_recorded[buf] = true;
  }
  c->n_cross += c->L.s.T;
  c->n_auto += c->L.s.T;
  return CORR_OK;
}

int corr_accumulate_autos(corr_ctx* c, const void* d_samples, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_accumulate_autos: NULL context");
  if (!d_samples) return fail(CORR_ERR_ARG, "corr_accumulate_autos: NULL samples");
  const bool tb = timer_begin(c, CORR_KERNEL_AUTOS, (cudaStream_t)stream);
  cudaError_t e = launch_autos(c->L.s, static_cast<const uint8_t*>(d_samples), c->L.s.T, c->d_autos, nullptr,
                               (cudaStream_t)stream);
  timer_end(c, CORR_KERNEL_AUTOS, (cudaStream_t)stream, tb);
  if (e != cudaSuccess) return cuda_fail(e, "corr_accumulate_autos: launch");
  c->n_auto += c->L.s.T;
  return CORR_OK;
}

int corr_reset(corr_ctx* c, int what, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_reset: NULL context");
  if (what < 1 || what > 3) return fail(CORR_ERR_ARG, "corr_reset: what must be CROSS, AUTO or both");
  cudaStream_t st = (cudaStream_t)stream;
  if (what & CORR_WHAT_CROSS) {
    cudaError_t e = cudaMemsetAsync(c->d_cross, 0, (size_t)c->L.cross_elems * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_soff, 0, (size_t)c->L.autos_elems * 16, st);
    if (e == cudaSuccess && c->d_cross_base) e = cudaMemsetAsync(c->d_cross_base, 0, (size_t)c->L.s.Bs * 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "corr_reset");
    c->n_cross = 0;
    c->n_off = 0;
  }
  if (what & CORR_WHAT_AUTO) {
    cudaError_t e = cudaMemsetAsync(c->d_autos, 0, (size_t)c->L.autos_elems * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_soff_auto, 0, (size_t)c->L.autos_elems * 16, st);
    if (e == cudaSuccess && c->d_auto_base) e = cudaMemsetAsync(c->d_auto_base, 0, (size_t)c->L.s.N * 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "corr_reset");
    c->n_auto = 0;
    c->n_off_auto = 0;
  }
  return CORR_OK;
}

int corr_dump(corr_ctx* c, void* out, int is_device_ptr, int what, int fmt, int reset, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_dump: NULL context");
  if (!out) return fail(CORR_ERR_ARG, "corr_dump: NULL output");
  if (what != CORR_WHAT_CROSS && what != CORR_WHAT_AUTO) return fail(CORR_ERR_ARG, "corr_dump: what must be CROSS or AUTO");
  if (fmt != CORR_FMT_CI64 && fmt != CORR_FMT_CF32 && fmt != CORR_FMT_CF32_NORM)
    return fail(CORR_ERR_ARG, "corr_dump: unknown format");
  cudaStream_t st = (cudaStream_t)stream;
  const long long* acc = what == CORR_WHAT_CROSS ? c->d_cross : c->d_autos;
  const long long n = what == CORR_WHAT_CROSS ? c->L.cross_elems : c->L.autos_elems;
  const long long ns = what == CORR_WHAT_CROSS ? c->n_cross : c->n_auto;
  const size_t esz = fmt == CORR_FMT_CI64 ? 8 : 4;
  Shape2 g;
  g.N = c->L.s.N;
  g.npol = c->L.s.npol;
  g.P = c->L.s.P;
  g.Bs = c->L.s.Bs;
  g.soff = what == CORR_WHAT_CROSS ? c->d_soff : c->d_soff_auto;
  g.t_off = what == CORR_WHAT_CROSS ? c->n_off : c->n_off_auto;
  g.autos = what == CORR_WHAT_AUTO ? 1 : 0;
  g.base = what == CORR_WHAT_CROSS ? c->d_cross_base : c->d_auto_base;
  cudaError_t e;
  if (is_device_ptr) {
    const bool tb = timer_begin(c, CORR_KERNEL_DUMP, st);
    e = launch_dump(acc, n, out, fmt, ns, 0, g, st);
    timer_end(c, CORR_KERNEL_DUMP, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "corr_dump: launch");
  } else {
    const long long per = (long long)(kStageBytes / esz) & ~1LL;  // whole (re, im) cells
    int buf = 0;
    for (long long k = 0; k < n; k += per) {
      const long long m = (n - k) < per ? (n - k) : per;
      const bool tb = timer_begin(c, CORR_KERNEL_DUMP, st);
      e = launch_dump(acc, m, c->d_stage[buf], fmt, ns, k, g, st);
      timer_end(c, CORR_KERNEL_DUMP, st, tb);
      if (e != cudaSuccess) return cuda_fail(e, "corr_dump: launch");
      e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + (size_t)k * esz, c->d_stage[buf], (size_t)m * esz,
                          cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_fail(e, "corr_dump: copy");
      buf ^= 1;
    }
  }
  if (reset) return corr_reset(c, what, stream);
  return CORR_OK;
}

int corr_dump_stations(corr_ctx* c, const int* stations, int n_stations, void* out, int is_device_ptr, int what,
                       int fmt, int reset, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_dump_stations: NULL context");
  if (!out || !stations) return fail(CORR_ERR_ARG, "corr_dump_stations: NULL output or station list");
  if (what != CORR_WHAT_CROSS && what != CORR_WHAT_AUTO)
    return fail(CORR_ERR_ARG, "corr_dump_stations: what must be CROSS or AUTO");
  if (fmt != CORR_FMT_CI64 && fmt != CORR_FMT_CF32 && fmt != CORR_FMT_CF32_NORM)
    return fail(CORR_ERR_ARG, "corr_dump_stations: unknown format");
  const int S = c->L.s.S;
  if (n_stations < 1 || n_stations > S) return fail(CORR_ERR_ARG, "corr_dump_stations: need 1..S stations");
  std::vector<char> seen((size_t)S, 0);
  for (int k = 0; k < n_stations; ++k) {
    const int a = stations[k];
    if (a < 0 || a >= S) return fail(CORR_ERR_ARG, "corr_dump_stations: station " + std::to_string(a) + " out of range");
    if (seen[(size_t)a]) return fail(CORR_ERR_ARG, "corr_dump_stations: station " + std::to_string(a) + " listed twice");
    seen[(size_t)a] = 1;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (n_stations > c->sel_cap) {
    int* d = nullptr;
    if (cudaMalloc(&d, (size_t)n_stations * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(CORR_ERR_OOM, "corr_dump_stations: station list allocation");
    }
    cudaStreamSynchronize(st);  // the old list may still be read by queued work on this stream
    cudaFree(c->d_sel);
    c->d_sel = d;
    c->sel_cap = n_stations;
  }
  long long** base = what == CORR_WHAT_CROSS ? &c->d_cross_base : &c->d_auto_base;
  const size_t base_bytes = (size_t)(what == CORR_WHAT_CROSS ? c->L.s.Bs : c->L.s.N) * 8;
  if (reset && !*base) {
    if (cudaMalloc(base, base_bytes) != cudaSuccess) {
      cudaGetLastError();
      *base = nullptr;
      return fail(CORR_ERR_OOM, "corr_dump_stations: sample-count allocation");
    }
    e = cudaMemsetAsync(*base, 0, base_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: sample-count init");
  }
  // pageable source: the call returns once the list has been staged, so `stations` may be reused
  e = cudaMemcpyAsync(c->d_sel, stations, (size_t)n_stations * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: station list upload");
  Shape2 g;
  g.N = c->L.s.N;
  g.npol = c->L.s.npol;
  g.P = c->L.s.P;
  g.Bs = c->L.s.Bs;
  g.soff = what == CORR_WHAT_CROSS ? c->d_soff : c->d_soff_auto;
  g.t_off = what == CORR_WHAT_CROSS ? c->n_off : c->n_off_auto;
  g.autos = what == CORR_WHAT_AUTO ? 1 : 0;
  g.base = *base;
  long long* acc = what == CORR_WHAT_CROSS ? c->d_cross : c->d_autos;
  const long long ns = what == CORR_WHAT_CROSS ? c->n_cross : c->n_auto;
  const size_t esz = fmt == CORR_FMT_CI64 ? 8 : 4;
  const size_t per_chan = (size_t)(what == CORR_WHAT_CROSS ? (long long)n_stations * (n_stations + 1) / 2 * g.P * 2
                                                           : (long long)n_stations * g.npol) * esz;
  const int C = c->L.s.C;
  if (is_device_ptr) {
    const bool tb = timer_begin(c, CORR_KERNEL_DUMP, st);
    e = launch_dump_select(acc, c->d_sel, n_stations, 0, C, out, fmt, ns, reset, g, st);
    timer_end(c, CORR_KERNEL_DUMP, st, tb);
    if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: launch");
  } else {
    const int nf_chunk = (int)(kStageBytes / per_chan);
    if (nf_chunk < 1) return fail(CORR_ERR_ARG, "corr_dump_stations: one channel exceeds the host staging buffer");
    int buf = 0;
    for (int f0 = 0; f0 < C; f0 += nf_chunk) {
      const int nf = C - f0 < nf_chunk ? C - f0 : nf_chunk;
      const bool tb = timer_begin(c, CORR_KERNEL_DUMP, st);
      e = launch_dump_select(acc, c->d_sel, n_stations, f0, nf, c->d_stage[buf], fmt, ns, reset, g, st);
      timer_end(c, CORR_KERNEL_DUMP, st, tb);
      if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: launch");
      e = cudaMemcpyAsync(static_cast<uint8_t*>(out) + (size_t)f0 * per_chan, c->d_stage[buf], (size_t)nf * per_chan,
                          cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: copy");
      buf ^= 1;
    }
  }
  if (reset) {
    e = launch_set_base(*base, c->d_sel, n_stations, ns, g, st);
    if (e != cudaSuccess) return cuda_fail(e, "corr_dump_stations: sample-count update");
  }
  return CORR_OK;
}

int corr_requantize(const void* d_in, int in_type, int n_inputs, int n_time, int n_pfb_chans, int chan0, int n_chans,
                    float gain, const float* d_gains, int symmetric, void* d_out, void* stream) {
  if (!d_in || !d_out) return fail(CORR_ERR_ARG, "corr_requantize: NULL buffer");
  if (in_type != CORR_IN_CI32 && in_type != CORR_IN_CF32) return fail(CORR_ERR_ARG, "corr_requantize: unknown input type");
  if ((reinterpret_cast<uintptr_t>(d_in) & 7) != 0 || (d_gains && (reinterpret_cast<uintptr_t>(d_gains) & 3) != 0))
    return fail(CORR_ERR_ARG, "corr_requantize: samples must be 8-byte and gains 4-byte aligned");
  if (n_inputs < 1 || n_time < 0 || n_pfb_chans < 1 || n_chans < 1 || chan0 < 0 || n_chans > 65535 ||
      (long long)chan0 + n_chans > n_pfb_chans)
    return fail(CORR_ERR_ARG, "corr_requantize: need 0 <= chan0, chan0 + n_chans <= n_pfb_chans, n_chans <= 65535");
  if (!(gain == gain)) return fail(CORR_ERR_ARG, "corr_requantize: gain is NaN");
  const cudaError_t e = launch_requant(d_in, in_type == CORR_IN_CI32 ? 0 : 1, n_inputs, n_time, n_pfb_chans, chan0,
                                       n_chans, gain, d_gains, symmetric != 0, static_cast<uint8_t*>(d_out),
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "corr_requantize: launch");
  return CORR_OK;
}

int corr_pfb_coeffs(int n_fft, int n_taps, int32_t* h_out) {
  if (!h_out) return fail(CORR_ERR_ARG, "corr_pfb_coeffs: NULL output");
  if (n_fft < 2 || (n_fft & (n_fft - 1)) != 0 || n_taps < 1 || n_taps > 64 || (long long)n_fft * n_taps > (1 << 24))
    return fail(CORR_ERR_ARG, "corr_pfb_coeffs: need n_fft a power of two >= 2 and 1 <= n_taps <= 64");
  const long long L = (long long)n_fft * n_taps;
  std::vector<double> h((size_t)L);
  double peak = 0.0;
  for (long long j = 0; j < L; ++j) {
    const double w = L > 1 ? 0.54 - 0.46 * std::cos(2.0 * M_PI * (double)j / (double)(L - 1)) : 1.0;  // Hamming
    const double u = ((double)j - 0.5 * (double)(L - 1)) / (double)n_fft;
    const double sinc = u == 0.0 ? 1.0 : std::sin(M_PI * u) / (M_PI * u);
    h[(size_t)j] = w * sinc;
    peak = std::fabs(h[(size_t)j]) > peak ? std::fabs(h[(size_t)j]) : peak;
  }
  const double scale = 131071.0 / peak;  // 18-bit signed coefficients, largest magnitude 2^17 - 1
  for (long long j = 0; j < L; ++j) h_out[j] = (int32_t)std::floor(h[(size_t)j] * scale + 0.5);
  return CORR_OK;
}

int corr_pfb(const int8_t* d_adc, int n_inputs, long long input_stride, long long n_samples, int n_taps,
             const int32_t* d_coeffs, int n_spectra, void* d_out, void* stream) {
  constexpr long long M = 8192;
  if (!d_adc || !d_coeffs || !d_out) return fail(CORR_ERR_ARG, "corr_pfb: NULL buffer");
  if (n_inputs < 1 || n_inputs > 65535 || n_taps < 1 || n_taps > 64 || n_spectra < 0 || n_spectra > (1 << 30))
    return fail(CORR_ERR_ARG, "corr_pfb: need 1 <= n_inputs <= 65535, 1 <= n_taps <= 64, n_spectra >= 0");
  if (((long long)n_spectra + n_taps - 1) * M > n_samples || n_samples > input_stride)
    return fail(CORR_ERR_ARG, "corr_pfb: need (n_spectra + n_taps - 1) * 8192 <= n_samples <= input_stride");
  if ((input_stride & 3) != 0 || (reinterpret_cast<uintptr_t>(d_adc) & 3) != 0 ||
      (reinterpret_cast<uintptr_t>(d_coeffs) & 15) != 0 || (reinterpret_cast<uintptr_t>(d_out) & 7) != 0)
    return fail(CORR_ERR_ARG, "corr_pfb: samples and stride 4-byte, coefficients 16-byte, output 8-byte aligned");
  const cudaError_t e = launch_pfb(d_adc, input_stride, n_inputs, n_spectra, n_taps, d_coeffs,
                                   static_cast<float2*>(d_out), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "corr_pfb: launch");
  return CORR_OK;
}

long long corr_samples_accumulated(const corr_ctx* c, int what) {
  if (!c) return CORR_ERR_ARG;
  if (what == CORR_WHAT_CROSS) return c->n_cross;
  if (what == CORR_WHAT_AUTO) return c->n_auto;
  return CORR_ERR_ARG;
}

int corr_sync(corr_ctx* c, void* stream) {
  if (!c) return fail(CORR_ERR_ARG, "corr_sync: NULL context");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "corr_sync");
  int flag = 0;
  e = cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "corr_sync: read error flag");
  if (flag != 0) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return fail(CORR_ERR_TIMEOUT, "corr_sync: a device-side wait timed out (code " + std::to_string(flag) + ")");
  }
  return CORR_OK;
}

int corr_profile_enable(corr_ctx* c, int on) {
  if (!c) return fail(CORR_ERR_ARG, "corr_profile_enable: NULL context");
  c->profiling = on != 0;
  return CORR_OK;
}

int corr_profile_read(corr_ctx* c, int kernel, double* total_ms, long long* launches) {
  if (!c) return fail(CORR_ERR_ARG, "corr_profile_read: NULL context");
  if (kernel < 0 || kernel >= CORR_KERNEL_COUNT) return fail(CORR_ERR_ARG, "corr_profile_read: unknown kernel id");
  KernelTimer& t = c->timers[kernel];
  drain_timer(t);
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.launches;
  t.ms = 0.0;
  t.launches = 0;
  return CORR_OK;
}

int corr_destroy(corr_ctx* c) {
  if (!c) return CORR_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_ctx(c);
  if (e != cudaSuccess) return cuda_fail(e, "corr_destroy: synchronize");
  return CORR_OK;
}

}  // extern "C"
