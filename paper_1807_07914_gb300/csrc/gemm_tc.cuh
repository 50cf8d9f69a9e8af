// BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32 accumulate in
// tensor memory:   C[M x N] = A[M x K] * B[N x K]^T   (both operands K-major).
//
// One CTA (4 warps) computes a 128 x 128 tile. K advances in steps of 64: all
// threads stage the A and B tiles into shared memory in the canonical
// no-swizzle core-matrix layout (two stages, so the next tile loads while the
// tensor core consumes the previous one); one elected thread issues four
// 128x128x16 MMAs per stage and commits them to the stage's mbarrier. Waits
// are bounded: a wait that runs out sets the error flag and every thread
// leaves the K loop together. The epilogue reads the accumulator with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows) and hands 32
// consecutive columns at a time to the epilogue functor.
#pragma once
#include "tc_util.cuh"

namespace tcg {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int TILE_BYTES = BM * BK * 2;              // 16 KB per operand per stage
constexpr int SMEM_BYTES = 4 * TILE_BYTES + 1024;    // 2 stages x (A, B) + alignment slack
constexpr uint32_t LBO = 128;                        // next core matrix along K
constexpr uint32_t SBO = 128 * (BK / 8);             // next 8-row group

// element (r, k) of a 128 x 64 tile -> byte offset of its 16-byte row chunk
__device__ __forceinline__ uint32_t tile_off(int r, int kv) {
  return (uint32_t)((r >> 3) * SBO + kv * LBO + (r & 7) * 16);
}

struct Operands {
  const uint16_t *A;  // BF16 bits, row r at A + r*lda
  const uint16_t *B;
  int M, N, K, lda, ldb;
  uint32_t *err;
};

__device__ __forceinline__ void stage_tile(uint8_t *dst, const uint16_t *src, int rows, int r0,
                                           int ld, int k0, int K) {
  // 128 rows x 8 vectors of 8 BF16 (16 bytes) each
  for (int v = threadIdx.x; v < BM * (BK / 8); v += blockDim.x) {
    const int r = v >> 3, kv = v & 7;
    const int gr = r0 + r, gk = k0 + kv * 8;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (gr < rows && gk < K) val = *reinterpret_cast<const uint4 *>(src + (int64_t)gr * ld + gk);
    *reinterpret_cast<uint4 *>(dst + tile_off(r, kv)) = val;
  }
}

// Epi: __device__ void operator()(int row, int col, const float (&v)[32]) const,
// called for columns col..col+31 of row `row` (row < M; columns may exceed N).
template <class Epi>
__global__ void __launch_bounds__(128) k_gemm_bf16(Operands op, Epi epi) {
  extern __shared__ uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                            ~(uintptr_t)1023);
  uint8_t *sA[2] = {sm, sm + TILE_BYTES};
  uint8_t *sB[2] = {sm + 2 * TILE_BYTES, sm + 3 * TILE_BYTES};
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, BN);  // 128 FP32 columns x 128 lanes
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_bf16(BM, BN);

  const int nk = (op.K + BK - 1) / BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt >= 2) {  // the MMAs that read this stage (tile kt-2) must be done
      const bool ok = tc::mbar_wait(&mbar[s], (uint32_t)(((kt - 2) >> 1) & 1));
      if (!ok) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
    stage_tile(sA[s], op.A, op.M, m0, op.lda, kt * BK, op.K);
    stage_tile(sB[s], op.B, op.N, n0, op.ldb, kt * BK, op.K);
    tc::fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA[s]), b0 = tc::smem_u32(sB[s]);
#pragma unroll
      for (int j = 0; j < BK / 16; ++j) {
        const uint64_t ad = tc::smem_desc(a0 + j * 2 * LBO, LBO, SBO);
        const uint64_t bd = tc::smem_desc(b0 + j * 2 * LBO, LBO, SBO);
        tc::mma_bf16(tmem, ad, bd, idesc, (kt > 0 || j > 0) ? 1u : 0u);
      }
      tc::mma_commit(&mbar[s]);
    }
  }
  // the last commit covers every MMA issued before it
  if (!s_fail && nk > 0) {
    const int last = nk - 1;
    const bool ok = tc::mbar_wait(&mbar[last & 1], (uint32_t)((last >> 1) & 1));
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  tc::fence_after_sync();
  if (!s_fail && nk > 0) {
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < BN; c += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (row < op.M && n0 + c < op.N) epi(row, n0 + c, v);
    }
  } else if (s_fail && threadIdx.x == 0 && op.err) {
    atomicOr(op.err, TNMPS_EFLAG_TIMEOUT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

template <class Epi>
inline cudaError_t launch(const Operands &op, const Epi &epi, cudaStream_t s) {
  if (op.M <= 0 || op.N <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<Epi>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((op.N + BN - 1) / BN, (op.M + BM - 1) / BM);
  k_gemm_bf16<Epi><<<grid, 128, SMEM_BYTES, s>>>(op, epi);
  return cudaGetLastError();
}

// plain FP32 store of C (row-major, ldc)
struct EpiStore {
  float *C;
  int N, ldc;
  __device__ void operator()(int row, int col, const float (&v)[32]) const {
    float *c = C + (int64_t)row * ldc + col;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (col + j < N) c[j] = v[j];
  }
};

}  // namespace tcg
