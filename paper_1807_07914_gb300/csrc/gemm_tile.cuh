// Shared-memory tiled complex GEMM core (CUDA cores, one output tile per CTA).
//
// C[i][j] = sum_k A(i,k) * B(k,j) for one batch entry. The operands are read
// through problem functors so that transposes, conjugation, Pauli actions on
// the physical index and ragged per-state bond dimensions are folded into the
// loads instead of being materialised.
#pragma once
#include "tnmps_internal.h"

template <typename R>
struct GemmCfg;
template <>
struct GemmCfg<double> {
  static constexpr int BM = 32, BN = 32, BK = 16;
};
template <>
struct GemmCfg<float> {
  static constexpr int BM = 64, BN = 64, BK = 16;
};

// Problem interface (device functions of P):
//   bool setup(int z, int &M, int &N, int &K)   -- per batch entry; false = skip
//   cx<R> a(int i, int k) const, cx<R> b(int k, int j) const
//   void store(int i, int j, cx<R> v) const
//   static constexpr bool A_KFAST, B_KFAST  -- k is the contiguous index
// One shared staging buffer for every instantiation of gemm_tile in a kernel
// (a __shared__ array inside the template would be allocated once per
// problem type).
constexpr int GEMM_SMEM_BYTES = 2 * 16 * 33 * 16;  // max over precisions of 2 BK (BM+1) sizeof
__device__ __forceinline__ unsigned char *gemm_smem() {
  __shared__ __align__(16) unsigned char buf[GEMM_SMEM_BYTES];
  return buf;
}

template <typename R, class P>
__device__ __forceinline__ void gemm_tile(P &p, int M, int N, int K, int i0, int j0) {
  constexpr int BM = GemmCfg<R>::BM, BN = GemmCfg<R>::BN, BK = GemmCfg<R>::BK;
  constexpr int TM = BM / 16, TN = BN / 16;
  static_assert(2 * BK * (BM + 1) * sizeof(cx<R>) <= GEMM_SMEM_BYTES, "gemm staging");
  typedef cx<R> RowA[BM + 1];
  typedef cx<R> RowB[BN + 1];
  RowA *As = reinterpret_cast<RowA *>(gemm_smem());
  RowB *Bs = reinterpret_cast<RowB *>(gemm_smem() + BK * (BM + 1) * sizeof(cx<R>));
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  cx<R> acc[TM][TN];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) acc[m][n] = mkc<R>(0, 0);

  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BK * BM; e += 256) {
      int kk, ii;
      if (P::A_KFAST) {
        kk = e % BK;
        ii = e / BK;
      } else {
        ii = e % BM;
        kk = e / BM;
      }
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < K) ? p.a(i, k) : mkc<R>(0, 0);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk, jj;
      if (P::B_KFAST) {
        kk = e % BK;
        jj = e / BK;
      } else {
        jj = e % BN;
        kk = e / BN;
      }
      const int j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < N && k < K) ? p.b(k, j) : mkc<R>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cx<R> av[TM], bv[TN];
#pragma unroll
      for (int m = 0; m < TM; ++m) av[m] = As[kk][ty + 16 * m];
#pragma unroll
      for (int n = 0; n < TN; ++n) bv[n] = Bs[kk][tx + 16 * n];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) cfma(acc[m][n], av[m], bv[n]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) {
      const int i = i0 + ty + 16 * m, j = j0 + tx + 16 * n;
      if (i < M && j < N) p.store(i, j, acc[m][n]);
    }
}

// complex64 operands, FP64 result: FP32 FMAs accumulate each BK-wide slice
// of K, and the slice sums are added in FP64. With |partial sums| bounded by
// the slice, the rounding stays ~BK u_32 |slice| per slice instead of the
// ~K u_32 |C| of a plain FP32 accumulation, at FP32 arithmetic speed.
// P::a/b return cx<float>; P::store takes cx<double>.
template <class P>
__device__ __forceinline__ void gemm_tile_mixed(P &p, int M, int N, int K, int i0, int j0) {
  constexpr int BM = GemmCfg<float>::BM, BN = GemmCfg<float>::BN, BK = GemmCfg<float>::BK;
  constexpr int TM = BM / 16, TN = BN / 16;
  static_assert(2 * BK * (BM + 1) * sizeof(cx<float>) <= GEMM_SMEM_BYTES, "gemm staging");
  typedef cx<float> RowA[BM + 1];
  typedef cx<float> RowB[BN + 1];
  RowA *As = reinterpret_cast<RowA *>(gemm_smem());
  RowB *Bs = reinterpret_cast<RowB *>(gemm_smem() + BK * (BM + 1) * sizeof(cx<float>));
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  cx<double> acc[TM][TN];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) acc[m][n] = mkc<double>(0, 0);

  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BK * BM; e += 256) {
      int kk, ii;
      if (P::A_KFAST) {
        kk = e % BK;
        ii = e / BK;
      } else {
        ii = e % BM;
        kk = e / BM;
      }
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < M && k < K) ? p.a(i, k) : mkc<float>(0, 0);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk, jj;
      if (P::B_KFAST) {
        kk = e % BK;
        jj = e / BK;
      } else {
        jj = e % BN;
        kk = e / BN;
      }
      const int j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < N && k < K) ? p.b(k, j) : mkc<float>(0, 0);
    }
    __syncthreads();
    cx<float> part[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TN; ++n) part[m][n] = mkc<float>(0, 0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cx<float> av[TM], bv[TN];
#pragma unroll
      for (int m = 0; m < TM; ++m) av[m] = As[kk][ty + 16 * m];
#pragma unroll
      for (int n = 0; n < TN; ++n) bv[n] = Bs[kk][tx + 16 * n];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) cfma(part[m][n], av[m], bv[n]);
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TN; ++n) {
        acc[m][n].re += (double)part[m][n].re;
        acc[m][n].im += (double)part[m][n].im;
      }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) {
      const int i = i0 + ty + 16 * m, j = j0 + tx + 16 * n;
      if (i < M && j < N) p.store(i, j, acc[m][n]);
    }
}

template <class P>
__global__ void __launch_bounds__(256) k_gemm_mixed(P p, int zbase) {
  int M, N, K;
  if (!p.setup((int)blockIdx.z + zbase, M, N, K)) return;
  const int i0 = blockIdx.y * GemmCfg<float>::BM, j0 = blockIdx.x * GemmCfg<float>::BN;
  if (i0 >= M || j0 >= N) return;
  gemm_tile_mixed(p, M, N, K, i0, j0);
}

template <class P>
static inline cudaError_t launch_gemm_mixed(const P &p, int Mmax, int Nmax, int entries,
                                            cudaStream_t s, uint64_t *launches = nullptr) {
  if (entries <= 0 || Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  for (int z0 = 0; z0 < entries; z0 += 65535) {
    const int nz = entries - z0 < 65535 ? entries - z0 : 65535;
    dim3 grid((Nmax + GemmCfg<float>::BN - 1) / GemmCfg<float>::BN,
              (Mmax + GemmCfg<float>::BM - 1) / GemmCfg<float>::BM, nz);
    k_gemm_mixed<P><<<grid, 256, 0, s>>>(p, z0);
    if (launches) ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Batched launch: grid (ceil(Nmax/BN), ceil(Mmax/BM), entries), 256 threads.
template <typename R, class P>
__global__ void __launch_bounds__(256) k_gemm(P p, int zbase) {
  int M, N, K;
  if (!p.setup((int)blockIdx.z + zbase, M, N, K)) return;
  const int i0 = blockIdx.y * GemmCfg<R>::BM, j0 = blockIdx.x * GemmCfg<R>::BN;
  if (i0 >= M || j0 >= N) return;
  gemm_tile<R>(p, M, N, K, i0, j0);
}

template <typename R, class P>
static inline cudaError_t launch_gemm(const P &p, int Mmax, int Nmax, int entries,
                                      cudaStream_t s, uint64_t *launches = nullptr) {
  if (entries <= 0 || Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  for (int z0 = 0; z0 < entries; z0 += 65535) {
    const int nz = entries - z0 < 65535 ? entries - z0 : 65535;
    dim3 grid((Nmax + GemmCfg<R>::BN - 1) / GemmCfg<R>::BN,
              (Mmax + GemmCfg<R>::BM - 1) / GemmCfg<R>::BM, nz);
    k_gemm<R, P><<<grid, 256, 0, s>>>(p, z0);
    if (launches) ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
