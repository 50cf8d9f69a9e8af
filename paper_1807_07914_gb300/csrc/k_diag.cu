// Diagnostic kernel of the failure-detection tests: a bounded device-side
// wait that runs out. Every wait of the tensor-core pipelines (bulk copies and
// MMAs tracked by mbarriers) gives up after a fixed number of SM clocks, raises
// the context's timeout flag and lets the kernel return, so a stall is
// reported by the host instead of hanging the GPU. This kernel exercises that
// path on purpose: it waits on a freshly initialised mbarrier phase that no
// thread ever completes (nothing is in flight on it), gives up after
// max_cycles and raises the same flag. No paper counterpart.
#include "tc_util.cuh"

namespace {

__global__ void k_debug_wait(uint32_t *err, long long max_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);  // one arrival expected; none will come
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, max_cycles)) atomicOr(err, TNMPS_EFLAG_TIMEOUT);
}

}  // namespace

cudaError_t launch_debug_wait(uint32_t *err, int64_t max_cycles, cudaStream_t s) {
  k_debug_wait<<<1, 32, 0, s>>>(err, (long long)max_cycles);
  return cudaGetLastError();
}
