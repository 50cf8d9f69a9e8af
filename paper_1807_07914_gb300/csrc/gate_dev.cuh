// CTA-level building blocks of the gate step (shared by the batched
// kernels, where a CTA handles one state of the batch, and the persistent
// multi-circuit kernel, where a CTA runs whole circuits).
#pragma once
#include "tnmps_internal.h"

namespace gdev {

// Theta = G X on the physical pair for elements e = start, start+stride, ...
// of the Dl x Dr grid; T row-major (2Dl) x (2Dr) in place, W its
// column-major copy (the Jacobi input).
template <typename R>
__device__ __forceinline__ void apply_gate4_range(const cx<R> *G, cx<R> *T, cx<R> *W, int Dl,
                                                  int Dr, int start, int stride) {
  const int M = 2 * Dl, N = 2 * Dr;
  for (int e = start; e < Dl * Dr; e += stride) {
    const int a = e / Dr, c = e - a * Dr;
    cx<R> x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = T[(int64_t)(2 * a + (q >> 1)) * N + (q & 1) * Dr + c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      cx<R> acc = mkc<R>(0, 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) cfma(acc, G[4 * r + q], x[q]);
      const int i = 2 * a + (r >> 1), j = (r & 1) * Dr + c;
      T[(int64_t)i * N + j] = acc;
      W[(int64_t)j * M + i] = acc;
    }
  }
}

// Truncation rule on the Jacobi output W (column-major M x N): singular
// values = column norms (FP64), stable descending order, keep those >=
// e_eff * ||sigma|| (and > 0), at most min(cap, M, N), at least one;
// A (M x k row-major) <- normalised kept columns. Returns k; *w = discarded
// weight of the step; *bad = non-finite or zero norm. Whole CTA.
template <typename R>
__device__ int select_cta(const cx<R> *W, int M, int N, int cap, double e_eff, cx<R> *A, double *w,
                          bool *bad) {
  __shared__ double sig[TNMPS_JACOBI_MAX_DIM];
  __shared__ int perm[TNMPS_JACOBI_MAX_DIM];
  __shared__ int s_k;
  __shared__ double s_w;
  __shared__ bool s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  for (int j = warp; j < N; j += nw) {
    double acc = 0;
    for (int r = lane; r < M; r += 32) {
      const cx<R> z = W[(int64_t)j * M + r];
      acc += (double)z.re * z.re + (double)z.im * z.im;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {  // stable descending rank
    const double sj = sig[j];
    int rank = 0;
    for (int i = 0; i < N; ++i) {
      const double si = sig[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0;
    for (int r = 0; r < N; ++r) total += sig[perm[r]] * sig[perm[r]];
    const double thr = e_eff * sqrt(total);
    int keep = 0;
    while (keep < N && sig[perm[keep]] >= thr && sig[perm[keep]] > 0) ++keep;
    int kmax = cap < M ? cap : M;
    kmax = kmax < N ? kmax : N;
    int k = keep < kmax ? keep : kmax;
    if (k < 1) k = 1;
    double dw = 0;
    for (int r = k; r < N; ++r) dw += sig[perm[r]] * sig[perm[r]];
    s_bad = !(total > 0) || !isfinite(total);
    s_w = s_bad ? 0.0 : dw / total;
    s_k = k;
  }
  __syncthreads();
  const int k = s_k;
  for (int e = threadIdx.x; e < M * k; e += blockDim.x) {
    const int i = e / k, r = e - i * k;
    const int j = perm[r];
    const double s = sig[j];
    const R inv = s > 0 ? (R)(1.0 / s) : R(0);
    const cx<R> z = W[(int64_t)j * M + i];
    A[e] = mkc<R>(z.re * inv, z.im * inv);
  }
  *w = s_w;
  *bad = s_bad;
  __syncthreads();
  return k;
}

// X (cnt elements) <- X / ||X||_F (FP64 sum). Whole CTA.
template <typename R>
__device__ void normalise_cta(cx<R> *X, int cnt) {
  __shared__ double red[32];
  double acc = 0;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x)
    acc += (double)X[e].re * X[e].re + (double)X[e].im * X[e].im;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double tot = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
  const R sc = tot > 0 ? (R)(1.0 / sqrt(tot)) : R(1);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) X[e] = mkc<R>(X[e].re * sc, X[e].im * sc);
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ R block_sum(R v, R *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Apply (I - f v v^H)-type updates column by column: for each column x of
// the trailing block, w = v^H x (warp reduction) and x -= coef * w * v. The
// reflector v sits in shared memory (vs, entries j..m-1, vs[j] = 1) and a
// warp keeps its column in registers between the dot and the update
// (m <= 32 * HR).
template <typename R, int HR>
__device__ __forceinline__ void reflect_columns(cx<R> *X, int ldx, int k0, int k1, int j, int m,
                                                const cx<R> *vs, cx<R> coef) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = k0 + warp; k < k1; k += nw) {
    cx<R> *x = X + (int64_t)k * ldx;
    cx<R> xr[HR];
    cx<R> w = mkc<R>(0, 0);
#pragma unroll
    for (int h = 0; h < HR; ++h) {
      const int i = j + lane + 32 * h;
      xr[h] = i < m ? x[i] : mkc<R>(0, 0);
      if (i < m) cfma(w, cconj(vs[i]), xr[h]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
      w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
    }
    const cx<R> f = cmul(coef, w);
#pragma unroll
    for (int h = 0; h < HR; ++h) {
      const int i = j + lane + 32 * h;
      if (i < m) {
        const cx<R> d = cmul(f, vs[i]);
        x[i] = mkc<R>(xr[h].re - d.re, xr[h].im - d.im);
      }
    }
  }
}

// In-place Householder QR of the column-major m x n matrix W (ld m):
// afterwards R is the upper triangle and the reflector vectors (v_j with
// implicit leading 1) sit below the diagonal; tau[j] holds their scalars
// (H_j = I - tau_j v_j v_j^H, A = H_0 ... H_{r-1} R). vs: shared scratch of
// m complex values. m <= 2 * TNMPS_MAX_CHI.
template <typename R>
__device__ void householder_qr(cx<R> *W, int m, int n, cx<R> *tau, R *red, cx<R> *vs) {
  const int r = m < n ? m : n;
  for (int j = 0; j < r; ++j) {
    cx<R> *col = W + (int64_t)j * m;
    R part = 0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x)
      part += col[i].re * col[i].re + col[i].im * col[i].im;
    const R xn2 = block_sum(part, red);
    const cx<R> alpha = col[j];
    __syncthreads();
    cx<R> tj = mkc<R>(0, 0);
    if (!(xn2 == R(0) && alpha.im == R(0))) {
      const R beta = -copysign(sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2), alpha.re);
      tj = mkc<R>((beta - alpha.re) / beta, -alpha.im / beta);
      // scal = 1 / (alpha - beta)
      const R dr = alpha.re - beta, di = alpha.im;
      const R den = dr * dr + di * di;
      const cx<R> sc = mkc<R>(dr / den, -di / den);
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
        const cx<R> v = cmul(col[i], sc);
        col[i] = v;
        vs[i] = v;
      }
      if (threadIdx.x == 0) {
        col[j] = mkc<R>(beta, 0);
        vs[j] = mkc<R>(1, 0);
      }
    }
    if (threadIdx.x == 0) tau[j] = tj;
    __syncthreads();
    if (tj.re == R(0) && tj.im == R(0)) continue;
    // columns k > j:  x <- x - conj(tau) v (v^H x)
    if (m <= 256) reflect_columns<R, 8>(W, m, j + 1, n, j, m, vs, cconj(tj));
    else reflect_columns<R, 16>(W, m, j + 1, n, j, m, vs, cconj(tj));
    __syncthreads();
  }
}

// Q = H_0 ... H_{r-1} [I; 0] (m x r, column-major ld m) from the reflectors in W.
template <typename R>
__device__ void householder_form_q(const cx<R> *W, int m, int n, const cx<R> *tau, cx<R> *Q,
                                   cx<R> *vs) {
  const int r = m < n ? m : n;
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int q = e / m, i = e - q * m;
    Q[e] = mkc<R>(i == q ? R(1) : R(0), 0);
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const cx<R> tj = tau[j];
    if (tj.re == R(0) && tj.im == R(0)) continue;
    const cx<R> *v = W + (int64_t)j * m;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) vs[i] = i == j ? mkc<R>(1, 0) : v[i];
    __syncthreads();
    if (m <= 256) reflect_columns<R, 8>(Q, m, j, r, j, m, vs, tj);
    else reflect_columns<R, 16>(Q, m, j, r, j, m, vs, tj);
    __syncthreads();
  }
}


// Right move core: C (2Dl x Dr row-major, in X) = Q R. X <- Q (Dl, 2, r);
// R stays in the upper triangle of W (column-major, ld 2Dl); Qbuf scratch.
// Returns r = min(2Dl, Dr). Whole CTA.
template <typename R>
__device__ int qr_right_cta(cx<R> *X, int Dl, int Dr, cx<R> *W, cx<R> *Qbuf) {
  const int m = 2 * Dl, n = Dr, r = m < n ? m : n;
  __shared__ cx<R> tau[2 * TNMPS_MAX_CHI];
  __shared__ cx<R> vs[2 * TNMPS_MAX_CHI];
  __shared__ R red[32];
  __syncthreads();
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int k = e / m, i = e - k * m;
    W[e] = X[(int64_t)i * n + k];
  }
  __syncthreads();
  householder_qr(W, m, n, tau, red, vs);
  householder_form_q(W, m, n, tau, Qbuf, vs);
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int i = e / r, q = e - i * r;
    X[e] = Qbuf[(int64_t)q * m + i];
  }
  __syncthreads();
  return r;
}

// Left move core: C (Dl x 2Dr row-major, in X) = L Q via QR of C^H = Q' R'.
// X <- Q'^H (r, 2, Dr); R' stays in W (column-major, ld 2Dr), L = R'^H.
// Returns r = min(2Dr, Dl). Whole CTA.
template <typename R>
__device__ int lq_left_cta(cx<R> *X, int Dl, int Dr, cx<R> *W, cx<R> *Qbuf) {
  const int m = 2 * Dr, n = Dl, r = m < n ? m : n;
  __shared__ cx<R> tau[2 * TNMPS_MAX_CHI];
  __shared__ cx<R> vs[2 * TNMPS_MAX_CHI];
  __shared__ R red[32];
  __syncthreads();
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) W[e] = cconj(X[e]);
  __syncthreads();
  householder_qr(W, m, n, tau, red, vs);
  householder_form_q(W, m, n, tau, Qbuf, vs);
  for (int e = threadIdx.x; e < r * m; e += blockDim.x) X[e] = cconj(Qbuf[e]);
  __syncthreads();
  return r;
}

}  // namespace gdev
