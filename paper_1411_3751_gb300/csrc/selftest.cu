// Failure detection without a fault: a one-thread kernel waits, with the bounded mbarrier wait that
// the tensor-core X-engines use for every pipeline handoff, on a barrier phase that nothing
// completes. When the limit passes it records `code` in the context's error word and returns; the
// next corr_sync reports CORR_ERR_TIMEOUT and clears the word, and the context stays usable.
#include "corr_internal.cuh"
#include "ptx_sm100.cuh"

namespace corr {
namespace {

__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns, int code) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  ptx::mbar_init(&bar, 1);  // one arrival completes phase 0; none ever comes
  ptx::fence_mbar_init();
  if (!ptx::mbar_wait(&bar, 0, limit_ns)) atomicCAS(err, 0, code);
}

}  // namespace

cudaError_t launch_wait_selftest(int* d_err, int limit_ms, int code, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(d_err, (unsigned long long)limit_ms * 1000000ull, code);
  return cudaGetLastError();
}

}  // namespace corr
