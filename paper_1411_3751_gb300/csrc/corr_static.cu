// corr_xengine_static: the tensor-path X-engine for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they correlate: code running inside a
// memory pool or arena owned by another runtime (a framework allocator, a real-time pipeline that
// forbids allocation after start-up, an embedding host that hands out only pre-sized buffers).
// This entry point keeps every byte of scratch it needs in one file-scope device array that exists
// from library load until process exit on every GPU that loads the library, and allocates nothing.
// The caller passes the input block and the output accumulators only.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "corr_internal.cuh"

namespace corr {
namespace {

// One shared scratch array (64 MiB, 256-byte aligned), carved per call as
//   [0, 256)                          error word of the bounded waits
//   [256, 256 + S)                    offset sums s[C][N][2] int64, S = round_up(16 C N, 256)
//   [.., .. + W)                      channel-major work list, W = round_up(24 C n_tiles, 256)
//   [.., .. + C T_pad R)              the e4m3 operand op[C][T_pad][R]
constexpr size_t kStaticScratchBytes = 64ull << 20;
constexpr size_t kOffSums = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per CUDA context (a device reset, or another
// context on the same device, loads the module again at another address), under a lock.
// Returns nullptr with *err set on failure.
void* scratch_address(std::string* err) {
  static std::mutex m;
  static std::map<unsigned long long, void*> by_context;
  const unsigned long long id = context_id();
  if (id == 0) {
    *err = "the current CUDA context cannot be identified";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(m);
  const auto it = by_context.find(id);
  if (it != by_context.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return nullptr;
  }
  by_context[id] = p;
  return p;
}

// Channel-major work list: item w = tile (w mod n_tiles) of channel w / n_tiles, the tiles being the
// plan-0 enumeration of the context path (a-side spans of 128 inputs, half-width on odd c-blocks).
__global__ void static_items_kernel(WorkItem* items, int N, int R, int n_tiles, long long n_items) {
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n_items; w += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(w / n_tiles);
    const int j = (int)(w % n_tiles);
    int k = 0;
    const int ncb = (N + 63) / 64;
    for (int cb = 0; cb < ncb; ++cb) {
      int a0 = 64 * cb;
      int nb = (cb & 1) ? 128 : 256;
      while (a0 < N) {
        if (2 * a0 + nb > R) nb = R - 2 * a0;
        if (k == j) {
          items[w] = WorkItem{0, f, 64 * cb, a0, nb, 0};
          cb = ncb;
          break;
        }
        ++k;
        a0 += nb / 2;
        nb = 256;
      }
    }
  }
}

// Adds the block's offset correction to every cross cell and every auto: the X-engine added the
// offset-domain Vu and Au for this block; V = Vu - (8 - 8i) s_a - (8 + 8i) conj(s_c) + 128 T and
// A = Au - 16 (Re s + Im s) + 128 T.
__global__ void static_correct_kernel(long long* __restrict__ cross, long long n_cells, long long* __restrict__ autos,
                                      long long n_autos, int N, int npol, long long Bs, const long long* __restrict__ s,
                                      long long T) {
  const int P = npol * npol;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_autos; k += (long long)gridDim.x * blockDim.x)
    autos[k] += -16 * (s[2 * k] + s[2 * k + 1]) + 128 * T;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < n_cells;
       cell += (long long)gridDim.x * blockDim.x) {
    const int pidx = (int)(cell % P);
    const long long fb = cell / P;
    const long long b = fb % Bs;
    const long long f = fb / Bs;
    long long sa = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (sa * (sa + 1) / 2 > b) --sa;
    while ((sa + 1) * (sa + 2) / 2 <= b) ++sa;
    const long long sc = b - sa * (sa + 1) / 2;
    const long long a = sa * npol + pidx / npol;
    const long long c = sc * npol + pidx % npol;
    const long long* s_a = s + (f * N + a) * 2;
    const long long* s_c = s + (f * N + c) * 2;
    cross[cell * 2] += -8 * (s_a[0] + s_a[1] + s_c[0] + s_c[1]) + 128 * T;
    cross[cell * 2 + 1] += -8 * (s_a[1] - s_a[0] + s_c[0] - s_c[1]);
  }
}

int static_fail(int code, const std::string& m) {
  set_last_error(m);
  return code;
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" int corr_xengine_static(const void* d_samples, int n_inputs, int n_chans, int n_time, int n_pol,
                                   long long* d_cross, long long* d_autos, void* cuda_stream) {
  if (!d_samples || !d_cross || !d_autos)
    return static_fail(CORR_ERR_ARG, "corr_xengine_static: NULL pointer");
  if (n_inputs < 1 || n_chans < 1 || n_time < 1 || (n_pol != 1 && n_pol != 2) || n_inputs % n_pol != 0 ||
      n_inputs > (1 << 16))
    return static_fail(CORR_ERR_ARG, "corr_xengine_static: invalid shape");
  const long long R = round_up(2LL * n_inputs, kF8RowAlign);
  const long long T_pad = round_up(n_time, kF8Kt);
  // tile count is a pure function of N (the context path's plan-0 enumeration, counted on the host)
  const int n_tiles = (int)f8_tile_plan(n_inputs, (int)R, 0).size();
  const long long n_items = (long long)n_tiles * n_chans;
  const size_t sums = (size_t)n_chans * n_inputs * 16;
  const size_t off_items = kOffSums + (size_t)round_up((long long)sums, 256);
  const size_t off_op = off_items + (size_t)round_up(n_items * (long long)sizeof(WorkItem), 256);
  const size_t need = off_op + (size_t)n_chans * (size_t)T_pad * (size_t)R;
  if (need > kStaticScratchBytes)
    return static_fail(CORR_ERR_ARG, "corr_xengine_static: needs " + std::to_string(need) +
                                         " bytes of scratch, above the fixed maximum of " +
                                         std::to_string(kStaticScratchBytes) +
                                         " (256 + round_up(16 C N, 256) + round_up(24 C n_tiles, 256) + "
                                         "C round_up(T, 128) round_up(2 N, 128))");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(CORR_ERR_CUDA, std::string("corr_xengine_static: ") + cudaGetErrorString(e));
  std::string aerr;
  unsigned char* base = static_cast<unsigned char*>(scratch_address(&aerr));
  if (!base) return static_fail(CORR_ERR_CUDA, "corr_xengine_static: " + aerr);
  int* d_err = reinterpret_cast<int*>(base);
  long long* d_s = reinterpret_cast<long long*>(base + kOffSums);
  WorkItem* d_items = reinterpret_cast<WorkItem*>(base + off_items);
  uint8_t* d_op = base + off_op;

  Shape sh;
  sh.N = n_inputs;
  sh.C = n_chans;
  sh.T = n_time;
  sh.npol = n_pol;
  sh.S = n_inputs / n_pol;
  sh.Bs = (long long)sh.S * (sh.S + 1) / 2;
  sh.P = n_pol * n_pol;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  CUtensorMap tmap;
  std::string err;
  if (encode_op_tensor_map(&tmap, d_op, (int)R, (int)T_pad, n_chans, &err) != 0)
    return static_fail(CORR_ERR_CUDA, "corr_xengine_static: " + err);

  // Everything that must start at zero for this call: the error flag and the offset sums.
  e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_s, 0, sums, st);
  if (e != cudaSuccess) return static_fail(CORR_ERR_CUDA, std::string("corr_xengine_static: ") + cudaGetErrorString(e));
  static_items_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, st>>>(d_items, n_inputs, (int)R, n_tiles, n_items);
  e = cudaGetLastError();
  const int T_run = (int)T_pad;
  if (e == cudaSuccess)
    e = launch_f8_prep(sh, static_cast<const uint8_t*>(d_samples), n_time, T_run, (int)T_pad, 0, (int)R, d_op, d_s,
                       nullptr, st);
  int num_sms = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (num_sms < 1) num_sms = 1;
  if (e == cudaSuccess)
  {
    XengArgs xa;
    std::memset(&xa, 0, sizeof(xa));
    xa.a[0].tmap = tmap;
    xa.a[0].cross = d_cross;
    xa.a[0].autos = d_autos;
    xa.a[0].Bs = sh.Bs;
    xa.a[0].N = n_inputs;
    xa.a[0].npol = n_pol;
    xa.items = d_items;
    xa.n_items = n_items;
    xa.T_run = T_run;
    xa.flush_len = kDefaultFlushF8;
    xa.err = d_err;
    e = launch_f8_xeng(xa, num_sms, st);
  }
  if (e == cudaSuccess) {
    const long long n_cells = (long long)n_chans * sh.Bs * sh.P;
    long long blocks = (n_cells + 255) / 256;
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    static_correct_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_cross, n_cells, d_autos, (long long)n_chans * n_inputs,
                                                            n_inputs, n_pol, sh.Bs, d_s, (long long)n_time);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return static_fail(CORR_ERR_CUDA, std::string("corr_xengine_static: ") + cudaGetErrorString(e));
  return CORR_OK;
}

extern "C" int corr_xengine_static_status(int* code, void* cuda_stream) {
  if (!code) return static_fail(CORR_ERR_ARG, "corr_xengine_static_status: NULL code");
  *code = 0;
  std::string aerr;
  unsigned char* base = static_cast<unsigned char*>(scratch_address(&aerr));
  if (!base) return static_fail(CORR_ERR_CUDA, "corr_xengine_static_status: " + aerr);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, base, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h != 0) e = cudaMemsetAsync(base, 0, sizeof(int), st);
  if (e == cudaSuccess && h != 0) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return static_fail(CORR_ERR_CUDA, std::string("corr_xengine_static_status: ") + cudaGetErrorString(e));
  *code = h;
  if (h != 0)
    return static_fail(CORR_ERR_TIMEOUT, "corr_xengine_static_status: a device-side wait timed out (code " +
                                             std::to_string(h) + ")");
  return CORR_OK;
}

extern "C" int corr_xengine_static_selftest_wait(int limit_ms, void* cuda_stream) {
  if (limit_ms < 1 || limit_ms > 2000)
    return static_fail(CORR_ERR_ARG, "corr_xengine_static_selftest_wait: limit_ms must be in [1, 2000]");
  std::string aerr;
  unsigned char* base = static_cast<unsigned char*>(scratch_address(&aerr));
  if (!base) return static_fail(CORR_ERR_CUDA, "corr_xengine_static_selftest_wait: " + aerr);
  const cudaError_t e = launch_wait_selftest(reinterpret_cast<int*>(base), limit_ms, 90, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess)
    return static_fail(CORR_ERR_CUDA, std::string("corr_xengine_static_selftest_wait: ") + cudaGetErrorString(e));
  return CORR_OK;
}
