// Self-test of the bounded waits of the step kernels (lcs_selftest_waits):
// each wait is run against a partner that never answers -- a predecessor
// tile that never publishes its look-back word, an mbarrier on which no copy
// ever completes -- and must give up after its iteration limit and report
// LCS_ERR_TIMEOUT instead of hanging.  Nothing here faults or traps.
#include "lcs.h"
#include "lcs_step_kernel.cuh"

namespace lcs {

// Limit of the mbarrier wait in the test (the step kernel uses PF_WAIT_LIMIT).
constexpr long long SELFTEST_MBAR_LIMIT = 1LL << 16;

// One warp.  status_arr[0] stays 0 (tile 0 never publishes); the warp
// resolves tile 1's prefix, which can only give up.  Then an mbarrier with
// one expected arrival that never comes is waited on with a bound.
__global__ void k_selftest_waits(unsigned long long *status_arr, int *lookback, int *mbar_out) {
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x & 31;
  resolve_prefix_warp(status_arr, 1, 0, 0ull, lookback);
  if (lane == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncwarp();
  if (lane == 0 && !mbar_wait(&bar, 0u, SELFTEST_MBAR_LIMIT)) *mbar_out = LCS_ERR_TIMEOUT;
}

}  // namespace lcs

extern "C" lcs_status lcs_selftest_waits(void *stream, int32_t *lookback, int32_t *mbarrier) {
  using namespace lcs;
  if (!lookback || !mbarrier) return LCS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *status_arr = nullptr;
  int *flags = nullptr;
  if (cudaMalloc((void **)&status_arr, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return LCS_ERR_CUDA;
  if (cudaMalloc((void **)&flags, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(status_arr);
    return LCS_ERR_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(status_arr, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) {
    k_selftest_waits<<<1, 32, 0, st>>>(status_arr, flags, flags + 1);
    e = cudaGetLastError();
  }
  int host[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, flags, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(status_arr);
  cudaFree(flags);
  if (e != cudaSuccess) return LCS_ERR_CUDA;
  *lookback = host[0];
  *mbarrier = host[1];
  return LCS_OK;
}
