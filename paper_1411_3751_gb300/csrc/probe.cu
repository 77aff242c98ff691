// Issue-rate probe of the tensor instruction the X-engine is built on: one CTA per SM issues
// tcgen05.mma kind::f8f6f4 (e4m3 operands, MN-major 128-byte-swizzled shared-memory tiles, M = 128,
// N = 128 or 256, K = 32, FP32 accumulation in TMEM) back to back from shared memory that never
// changes, so no operand traffic, barrier or epilogue limits it. The rate it reports is the ceiling
// of a single-SM tcgen05 X-engine on this GPU at the clock the GPU runs at; the benchmark reports
// the X-engine against it beside the measured bf16 peak.
#include <algorithm>
#include <string>
#include <vector>

#include "corr_internal.cuh"
#include "ptx_sm100.cuh"

namespace corr {
namespace {

constexpr int kProbeA = 128 * 128;             // 128 rows x 128 samples (four K = 32 slices)
constexpr int kProbeB = 2 * 128 * 128;         // two 128-row atoms
constexpr int kProbeSmem = 120 * 1024;         // more than half an SM's shared memory: one CTA per SM
constexpr uint64_t kProbeWaitNs = 2000000000ull;

__global__ void __launch_bounds__(128, 1) mma_rate_kernel(int n_mma, int n_cols, unsigned long long* cycles,
                                                          int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kProbeA + kProbeB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5;
  // operands: zeros (any finite e4m3 bytes give the same rate)
  for (int i = threadIdx.x; i < (kProbeA + kProbeB) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  ptx::fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    ptx::mbar_init(bar, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(tslot, 256);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tbase = *tslot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = ptx::idesc_f8_e4m3(128, n_cols, 1, 1);
    const uint32_t a_addr = ptx::smem_u32(smem), b_addr = a_addr + kProbeA;
    const long long t0 = clock64();
    for (int i = 0; i < n_mma; ++i) {
      const int kk = i & 3;
      const uint64_t ad = ptx::smem_desc(a_addr + kk * 4096, 16, 1024, 2);
      const uint64_t bd = ptx::smem_desc(b_addr + kk * 4096, kProbeB / 2, 1024, 2);
      ptx::mma_f8f6f4(tbase, ad, bd, idesc, i > 0 ? 1u : 0u);
    }
    ptx::mma_commit(bar);
    const bool ok = ptx::mbar_wait(bar, 0, kProbeWaitNs);
    const long long t1 = clock64();
    cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
    if (!ok) {
      atomicCAS(err, 0, 1);
      // the MMAs need nothing to complete: give them the time they take before TMEM is released
      ptx::mbar_wait(bar, 0, kProbeWaitNs);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tbase, 256);
}

}  // namespace
}  // namespace corr

using namespace corr;

extern "C" int corr_probe_mma_rate(int n_mma, int n_cols, double* tflops, double* cycles_per_mma, void* cuda_stream) {
  if (n_mma < 1 || n_mma > (1 << 20) || (n_cols != 128 && n_cols != 256)) {
    set_last_error("corr_probe_mma_rate: need 1 <= n_mma <= 2^20 and n_cols 128 or 256");
    return CORR_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = set_smem_limit(reinterpret_cast<const void*>(mma_rate_kernel), kProbeSmem);
  if (e != cudaSuccess) {
    set_last_error(std::string("corr_probe_mma_rate: ") + cudaGetErrorString(e));
    return CORR_ERR_CUDA;
  }
  unsigned long long* d_cycles = nullptr;
  int* d_err = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<unsigned long long> cyc((size_t)sms);
  int h_err = 0;
  float ms = 0.f;
  e = cudaMalloc(&d_cycles, sizeof(unsigned long long) * (size_t)sms);
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  // the first launch warms up (instruction cache, TMEM allocator); the second is timed
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    if (rep == 1) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) {
      mma_rate_kernel<<<sms, 128, kProbeSmem, st>>>(n_mma, n_cols, d_cycles, d_err);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && rep == 1) e = cudaEventRecord(ev[1], st);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  if (e == cudaSuccess)
    e = cudaMemcpy(cyc.data(), d_cycles, sizeof(unsigned long long) * (size_t)sms, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_cycles);
  cudaFree(d_err);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) {
    set_last_error(std::string("corr_probe_mma_rate: ") + cudaGetErrorString(e));
    return CORR_ERR_CUDA;
  }
  if (h_err != 0) {
    set_last_error("corr_probe_mma_rate: the completion wait timed out");
    return CORR_ERR_TIMEOUT;
  }
  std::sort(cyc.begin(), cyc.end());
  const double flops = 2.0 * 128.0 * (double)n_cols * 32.0 * (double)n_mma * (double)sms;
  if (tflops) *tflops = ms > 0.f ? flops / ((double)ms * 1e-3) / 1e12 : 0.0;
  if (cycles_per_mma) *cycles_per_mma = (double)cyc[cyc.size() / 2] / (double)n_mma;
  return CORR_OK;
}
