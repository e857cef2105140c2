// Self-test of the bounded device waits (wlr_selftest_bounded_wait): the tensor-core
// kernels wait on mbarriers with a time limit, after which they record an error bit and
// return instead of hanging.  This kernel runs that same wait on a barrier that nothing
// ever completes, so the limit always runs out; nothing else is in flight (no copy, no
// MMA, no tensor memory), so the kernel simply returns with the bit set.
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/wlr.h"
#include "wlr_tc.cuh"

namespace {

__global__ void wait_on_nothing(unsigned long long limit_ns, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    wlr::tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !wlr::tc::mbar_wait(&bar, 0u, limit_ns)) atomicOr(err, wlr::tc::ERRBIT_TIMEOUT);
}

}  // namespace

extern "C" wlr_status wlr_selftest_bounded_wait(int64_t limit_ns, void* cuda_stream) {
  if (limit_ns < 1 || limit_ns > 2000000000LL) {
    wlr::set_global_error("limit_ns must be in [1, 2e9]");
    return WLR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* err = nullptr;
  int h = 0;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    wlr::set_global_error("cudaMalloc failed");
    return WLR_ERR_OOM;
  }
  wlr_status out = WLR_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) out = WLR_ERR_CUDA;
  if (out == WLR_OK) {
    wait_on_nothing<<<1, 32, 0, st>>>((unsigned long long)limit_ns, err);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      out = WLR_ERR_CUDA;
  }
  cudaFree(err);
  if (out != WLR_OK) {
    wlr::set_global_error("CUDA call failed in the bounded-wait self-test");
    return out;
  }
  if (h & wlr::tc::ERRBIT_TIMEOUT) {
    wlr::set_global_error("the bounded wait gave up as designed");
    return WLR_ERR_DEVICE_TIMEOUT;
  }
  wlr::set_global_error("");
  return WLR_OK;
}
