// ALU ceiling of the GPU: the issue rate of fused multiply-adds on the CUDA
// cores in FP32 and FP64. The Jacobi SVD (K3) is bound by these pipes, so its
// roofline fraction is taken against this measured rate rather than a
// nominal or derived figure. No paper counterpart: measurement only.
//
// Every thread runs CH independent FMA chains (enough to cover the pipe
// latency at full occupancy); the operands are kernel arguments, so nothing
// folds at compile time, and the chains' sum is stored so nothing is dead.
#include "tnmps_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T *sink, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  sink[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" tnmps_status tnmps_alu_peak_dev(int bits, int blocks, int iters, void *sink_dev,
                                           double *flops, void *stream) {
  if ((bits != 32 && bits != 64) || blocks < 1 || iters < 1 || !sink_dev) return TNMPS_ERR_ARG;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (bits == 32)
    k_fma_peak<float><<<blocks, kThreads, 0, s>>>(static_cast<float *>(sink_dev), 0.999f, 1e-3f,
                                                  iters);
  else
    k_fma_peak<double><<<blocks, kThreads, 0, s>>>(static_cast<double *>(sink_dev), 0.999, 1e-3,
                                                   iters);
  if (cudaGetLastError() != cudaSuccess) return TNMPS_ERR_CUDA;
  if (flops)
    *flops = 2.0 * (double)blocks * kThreads * (double)iters * kUnroll * kChains;
  return TNMPS_OK;
}
