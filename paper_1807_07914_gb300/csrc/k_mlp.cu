// Tensor-core GEMM entry point (tcgen05, BF16 in / FP32 out).
#include "gemm_tc.cuh"
#include "tnmps_internal.h"

extern "C" tnmps_status tnmps_gemm_bf16_dev(int M, int N, int K, const uint16_t *A, int lda,
                                           const uint16_t *B, int ldb, float *C, int ldc,
                                           void *stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || (K % 8) || (lda % 8) || (ldb % 8) ||
      lda < K || ldb < K || ldc < N || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return TNMPS_ERR_ARG;
  tcg::Operands op{A, B, M, N, K, lda, ldb, nullptr};
  tcg::EpiStore epi{C, N, ldc};
  cudaError_t e = tcg::launch(op, epi, (cudaStream_t)stream);
  return e == cudaSuccess ? TNMPS_OK : TNMPS_ERR_CUDA;
}
