// CTA-level building blocks of the gate step (shared by the batched
// kernels, where a CTA handles one state of the batch, and the persistent
// multi-circuit kernel, where a CTA runs whole circuits).
#pragma once
#include "tnmps_internal.h"

namespace gdev {

// Theta = G X on the physical pair for elements e = start, start+stride, ...
// of the Dl x Dr grid; T row-major (2Dl) x (2Dr) in place, W (unless null)
// its column-major copy (the Jacobi input on Theta itself).
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
      if (W) W[(int64_t)j * M + i] = acc;
    }
  }
}

// Truncation rule on the Jacobi output W (column-major M x N): singular
// values = column norms (FP64), stable descending order, keep those >=
// e_eff * ||sigma|| (and > 0), at most min(cap, M, N), at least one;
// A (M x k row-major) <- normalised kept columns. Returns k; *w = discarded
// weight of the step; *bad = non-finite or zero norm. Whole CTA. A lane sums
// its share of a column in R (FP32 for complex64: the columns carry FP32
// rounding already), the warp reduction runs in FP64.
template <typename R>
__device__ int select_cta(const cx<R> *W, int M, int N, int cap, double e_eff, cx<R> *A, double *w,
                          bool *bad) {
  __shared__ double sig[TNMPS_JACOBI_MAX_DIM];
  __shared__ int perm[TNMPS_JACOBI_MAX_DIM];
  __shared__ R inv_s[TNMPS_JACOBI_MAX_DIM];  // 1 / sigma of the kept column of rank r
  __shared__ int s_k;
  __shared__ double s_w;
  __shared__ bool s_bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  for (int j = warp; j < N; j += nw) {
    R part = 0;
    for (int r = lane; r < M; r += 32) {
      const cx<R> z = W[(int64_t)j * M + r];
      part = fma(z.re, z.re, fma(z.im, z.im, part));
    }
    double acc = (double)part;
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
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const double s = sig[perm[r]];
    inv_s[r] = s > 0 ? (R)(1.0 / s) : R(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * k; e += blockDim.x) {
    const int i = e / k, r = e - i * k;
    const R inv = inv_s[r];
    const cx<R> z = W[(int64_t)perm[r] * M + i];
    A[e] = mkc<R>(z.re * inv, z.im * inv);
  }
  *w = s_w;
  *bad = s_bad;
  __syncthreads();
  return k;
}

// X (cnt elements) <- X / ||X||_F (FP64 sum of R partial sums over runs of 8
// elements). Whole CTA.
template <typename R>
__device__ void normalise_cta(cx<R> *X, int cnt) {
  __shared__ double red[32];
  double acc = 0;
  // runs of 8 of a thread's elements summed in R, the runs in FP64
  for (int e0 = threadIdx.x; e0 < cnt; e0 += 8 * blockDim.x) {
    R part = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < cnt) part = fma(X[e].re, X[e].re, fma(X[e].im, X[e].im, part));
    }
    acc += (double)part;
  }
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
// (m <= 32 * HR). Row i of column k sits at X[k * ldx + i - roff].
template <typename R, int HR>
__device__ __forceinline__ void reflect_columns(cx<R> *X, int ldx, int k0, int k1, int j, int m,
                                                const cx<R> *vs, cx<R> coef, int roff = 0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = k0 + warp; k < k1; k += nw) {
    cx<R> *x = X + (int64_t)k * ldx - roff;
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
// ------------------------------------------------ blocked (compact WY) form
// The reflectors j0..j0+nb-1 of a panel combine into H_j0 ... H_{j0+nb-1} =
// I - V T V^H (T upper triangular, nb x nb; column k of V is v_{j0+k}: 1 on
// row j0+k, W below it, 0 above). Applying a panel's block reflector reads each
// target column once per panel instead of once per reflector.

// v_{j0+k}[i] from the factored W (ld ldw)
template <typename R>
__device__ __forceinline__ cx<R> vrow(const cx<R> *W, int ldw, int j0, int k, int i) {
  const int d = j0 + k;
  return i > d ? W[(int64_t)d * ldw + i] : mkc<R>(i == d ? R(1) : R(0), R(0));
}

// Sum K per-lane values over the warp; every lane receives all K sums
// (halving exchanges, then a broadcast from the lane that holds each sum).
template <typename R, int K>
__device__ __forceinline__ void warp_allsum(R *v, int lane) {
  static_assert(K == 8 || K == 16 || K == 32, "warp_allsum width");
  R w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = v[k];
  int n = K;
#pragma unroll
  for (int o = 16; o >= 32 / K; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < K / 2; ++k) {
      if (k < n / 2) {
        const R keep = hi ? w[k + n / 2] : w[k];
        const R send = hi ? w[k] : w[k + n / 2];
        w[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    n >>= 1;
  }
  R t = w[0];
#pragma unroll
  for (int o = 16 / K; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = __shfl_sync(0xffffffffu, t, (32 / K) * k);
}

// Stage the panel's reflectors in shared memory: Vs[k * VLD + (i - j0)] =
// v_{j0+k}[i] for rows j0 <= i < j0 + VLD (explicit 1 and zeros), k < NB
// (columns k >= nb zero).
template <typename R, int NB, int VLD>
__device__ void stage_panel(const cx<R> *W, int ldw, int j0, int nb, int m, cx<R> *Vs) {
  for (int e = threadIdx.x; e < NB * VLD; e += blockDim.x) {
    const int k = e / VLD, i = j0 + (e - k * VLD);
    Vs[e] = (k < nb && i < m) ? vrow(W, ldw, j0, k, i) : mkc<R>(0, 0);
  }
  __syncthreads();
}

// T of the staged panel into Ts (NB x NB row-major, smem): T[k][k] = tau_k,
// T[0:k, k] = -tau_k T[0:k, 0:k] (V[:, 0:k]^H v_k). Gs: NB x NB smem scratch.
template <typename R, int NB, int VLD>
__device__ void block_tfactor(const cx<R> *Vs, int j0, int nb, int m, const cx<R> *tau, cx<R> *Ts,
                              cx<R> *Gs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int rows = m - j0 < VLD ? m - j0 : VLD;
  for (int p = warp; p < nb * nb; p += nw) {
    const int i = p / nb, k = p - i * nb;
    if (i >= k) continue;
    cx<R> acc = mkc<R>(0, 0);
    for (int row = k + lane; row < rows; row += 32)
      cfma(acc, cconj(Vs[i * VLD + row]), Vs[k * VLD + row]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) Gs[i * NB + k] = acc;
  }
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < NB; ++k) {
      cx<R> val = mkc<R>(0, 0);
      if (k < nb && lane < k) {
        for (int l = lane; l < k; ++l) cfma(val, Ts[lane * NB + l], Gs[l * NB + k]);
        val = cmul(mkc<R>(-tau[j0 + k].re, -tau[j0 + k].im), val);
      }
      __syncwarp();
      if (lane < NB) {
        cx<R> out = mkc<R>(0, 0);
        if (k < nb) out = lane < k ? val : (lane == k ? tau[j0 + k] : mkc<R>(0, 0));
        Ts[lane * NB + k] = out;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// Columns k0..k1-1 of X (ld ldx): x <- (I - V op(T) V^H) x with op(T) = T^H
// (herm: the QR trailing update, H^H of each reflector in order) or T (forming
// Q). Only rows >= j0 change. A warp takes two columns at a time, both in
// registers (m - j0 <= 32 HR), so each staged reflector value read from
// shared memory serves two columns.
template <typename R, int HR, int NB>
__device__ void apply_block_reflector(cx<R> *X, int ldx, int k0, int k1, const cx<R> *Vs,
                                      int j0, int m, const cx<R> *Ts, bool herm) {
  constexpr int VLD = 32 * HR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int col = k0 + 2 * warp; col < k1; col += 2 * nw) {
    const bool two = col + 1 < k1;
    cx<R> *x0 = X + (int64_t)col * ldx;
    cx<R> *x1 = x0 + ldx;
    cx<R> xr[2][HR];
    R w[4 * NB];  // column 0: w[0 .. 2NB), column 1: w[2NB .. 4NB)
#pragma unroll
    for (int k = 0; k < 4 * NB; ++k) w[k] = R(0);
#pragma unroll
    for (int h = 0; h < HR; ++h) {
      const int i = j0 + lane + 32 * h;
      xr[0][h] = i < m ? x0[i] : mkc<R>(0, 0);
      xr[1][h] = (two && i < m) ? x1[i] : mkc<R>(0, 0);
      if (i < m) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const cx<R> v = Vs[k * VLD + lane + 32 * h];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            R *wq = w + 2 * NB * q;
            wq[2 * k] = fma(v.re, xr[q][h].re, fma(v.im, xr[q][h].im, wq[2 * k]));
            wq[2 * k + 1] = fma(v.re, xr[q][h].im, fma(-v.im, xr[q][h].re, wq[2 * k + 1]));
          }
        }
      }
    }
    warp_allsum<R, 4 * NB>(w, lane);
    // w <- op(T) w in place: T upper (rows ascending), T^H lower (rows descending)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      R *wq = w + 2 * NB * q;
      if (herm) {
#pragma unroll
        for (int i = NB - 1; i >= 0; --i) {
          cx<R> a = mkc<R>(0, 0);
#pragma unroll
          for (int k = 0; k <= i; ++k)
            cfma(a, cconj(Ts[k * NB + i]), mkc<R>(wq[2 * k], wq[2 * k + 1]));
          wq[2 * i] = a.re;
          wq[2 * i + 1] = a.im;
        }
      } else {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
          cx<R> a = mkc<R>(0, 0);
#pragma unroll
          for (int k = i; k < NB; ++k) cfma(a, Ts[i * NB + k], mkc<R>(wq[2 * k], wq[2 * k + 1]));
          wq[2 * i] = a.re;
          wq[2 * i + 1] = a.im;
        }
      }
    }
#pragma unroll
    for (int h = 0; h < HR; ++h) {
      const int i = j0 + lane + 32 * h;
      if (i < m) {
        cx<R> a0 = xr[0][h], a1 = xr[1][h];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
          const cx<R> v = Vs[k * VLD + lane + 32 * h];
          a0.re -= v.re * w[2 * k] - v.im * w[2 * k + 1];
          a0.im -= v.re * w[2 * k + 1] + v.im * w[2 * k];
          a1.re -= v.re * w[2 * NB + 2 * k] - v.im * w[2 * NB + 2 * k + 1];
          a1.im -= v.re * w[2 * NB + 2 * k + 1] + v.im * w[2 * NB + 2 * k];
        }
        x0[i] = a0;
        if (two) x1[i] = a1;
      }
    }
  }
}

// householder_qr with panels of NB reflectors: each panel is factored with
// the reflector-at-a-time loop restricted to its own columns, then its block
// reflector updates the trailing columns once. Same factorisation as
// householder_qr (up to summation order). Panel factorisation: warp w keeps
// panel column j0 + w in registers (the CTA has at least NB warps); warp k
// forms reflector j0 + k from its column with a warp reduction and writes it
// as column k of the staged panel Vs (0 above its row, 1 on it, the scaled
// column below), and after one barrier the warps of the later columns apply it
// in registers. The factored columns then go back to W, and Vs is already the
// staged panel of the trailing update.
template <typename R, int NB, int HR>
__device__ void householder_qr_blocked(cx<R> *W, int m, int n, cx<R> *tau, R *red, cx<R> *vs,
                                       cx<R> *Ts, cx<R> *Gs, cx<R> *Vs) {
  constexpr int VLD = 32 * HR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = m < n ? m : n;
  for (int j0 = 0; j0 < r; j0 += NB) {
    const int nb = r - j0 < NB ? r - j0 : NB;
    const bool own = warp < nb;
    const int jc = j0 + warp;  // this warp's panel column
    cx<R> xr[HR];              // rows j0 + lane + 32 h
#pragma unroll
    for (int h = 0; h < HR; ++h) {
      const int i = j0 + lane + 32 * h;
      xr[h] = (own && i < m) ? W[(int64_t)jc * m + i] : mkc<R>(0, 0);
    }
    for (int k = 0; k < nb; ++k) {
      const int j = j0 + k;
      cx<R> *vk = Vs + k * VLD;  // v_j, row i at vk[i - j0]
      if (warp == k) {
        R part = 0;
#pragma unroll
        for (int h = 0; h < HR; ++h) {
          const int i = j0 + lane + 32 * h;
          if (i > j && i < m) part = fma(xr[h].re, xr[h].re, fma(xr[h].im, xr[h].im, part));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const R xn2 = part;
        // row j is held by lane k, register 0 (k < NB <= 32)
        const cx<R> alpha = mkc<R>(__shfl_sync(0xffffffffu, xr[0].re, k),
                                   __shfl_sync(0xffffffffu, xr[0].im, k));
        cx<R> tj = mkc<R>(0, 0);
        if (!(xn2 == R(0) && alpha.im == R(0))) {
          const R beta =
              -copysign(sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2), alpha.re);
          tj = mkc<R>((beta - alpha.re) / beta, -alpha.im / beta);
          const R dr = alpha.re - beta, di = alpha.im;
          const R den = dr * dr + di * di;
          const cx<R> sc = mkc<R>(dr / den, -di / den);  // 1 / (alpha - beta)
#pragma unroll
          for (int h = 0; h < HR; ++h) {
            const int i = j0 + lane + 32 * h;
            if (i > j && i < m) xr[h] = cmul(xr[h], sc);
          }
          if (lane == k) xr[0] = mkc<R>(beta, 0);
        }
#pragma unroll
        for (int h = 0; h < HR; ++h) {
          const int i = j0 + lane + 32 * h;
          if (i < m) vk[i - j0] = i > j ? xr[h] : mkc<R>(i == j ? R(1) : R(0), R(0));
        }
        if (lane == 0) tau[j] = tj;
      }
      __syncthreads();
      const cx<R> tj = tau[j];
      if (own && warp > k && !(tj.re == R(0) && tj.im == R(0))) {
        // x <- H_j^H x = x - conj(tau_j) v (v^H x)
        cx<R> w = mkc<R>(0, 0);
#pragma unroll
        for (int h = 0; h < HR; ++h) {
          const int i = j0 + lane + 32 * h;
          if (i < m) cfma(w, cconj(vk[i - j0]), xr[h]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
          w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
        }
        const cx<R> f = cmul(cconj(tj), w);
#pragma unroll
        for (int h = 0; h < HR; ++h) {
          const int i = j0 + lane + 32 * h;
          if (i < m) {
            const cx<R> d = cmul(f, vk[i - j0]);
            xr[h] = mkc<R>(xr[h].re - d.re, xr[h].im - d.im);
          }
        }
      }
    }
    // R on and above the diagonal, the reflectors below it
    if (own) {
#pragma unroll
      for (int h = 0; h < HR; ++h) {
        const int i = j0 + lane + 32 * h;
        if (i < m) W[(int64_t)jc * m + i] = xr[h];
      }
    }
    for (int e = threadIdx.x; e < (NB - nb) * VLD; e += blockDim.x) Vs[nb * VLD + e] = mkc<R>(0, 0);
    __syncthreads();
    if (j0 + nb >= n) continue;
    block_tfactor<R, NB, VLD>(Vs, j0, nb, m, tau, Ts, Gs);
    apply_block_reflector<R, HR, NB>(W, m, j0 + nb, n, Vs, j0, m, Ts, true);
    __syncthreads();
  }
}

// householder_form_q with the block reflectors of NB-wide panels, last panel first.
template <typename R, int NB, int HR>
__device__ void householder_form_q_blocked(const cx<R> *W, int m, int n, const cx<R> *tau,
                                           cx<R> *Q, cx<R> *Ts, cx<R> *Gs, cx<R> *Vs) {
  const int r = m < n ? m : n;
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int q = e / m, i = e - q * m;
    Q[e] = mkc<R>(i == q ? R(1) : R(0), 0);
  }
  __syncthreads();
  for (int j0 = ((r - 1) / NB) * NB; j0 >= 0; j0 -= NB) {
    const int nb = r - j0 < NB ? r - j0 : NB;
    stage_panel<R, NB, 32 * HR>(W, m, j0, nb, m, Vs);
    block_tfactor<R, NB, 32 * HR>(Vs, j0, nb, m, tau, Ts, Gs);
    apply_block_reflector<R, HR, NB>(Q, m, j0, r, Vs, j0, m, Ts, false);
    __syncthreads();
  }
}

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
// Returns r = min(2Dl, Dr). Whole CTA. HR > 0: panels of NB reflectors staged
// in shared memory and applied as block reflectors, 2 Dl <= 32 HR (one
// reflector at a time when the staged panel does not fit the static shared
// memory: complex128 with HR = 16); HR = 0: one reflector at a time.
template <typename R, int HR = 0, int NB = sizeof(R) == 4 ? 8 : 4>
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
  // staged panel + tau/vs arrays within 40 KB of static shared memory
  if constexpr (HR > 0 &&
                (NB * 32 * HR + 4 * TNMPS_MAX_CHI) * sizeof(cx<R>) <= 40960) {
    __shared__ cx<R> Ts[NB * NB], Gs[NB * NB];
    __shared__ __align__(16) cx<R> Vs[NB * 32 * HR];  // the panel's reflectors
    householder_qr_blocked<R, NB, HR>(W, m, n, tau, red, vs, Ts, Gs, Vs);
    householder_form_q_blocked<R, NB, HR>(W, m, n, tau, Qbuf, Ts, Gs, Vs);
  } else {
    householder_qr(W, m, n, tau, red, vs);
    householder_form_q(W, m, n, tau, Qbuf, vs);
  }
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int i = e / r, q = e - i * r;
    X[e] = Qbuf[(int64_t)q * m + i];
  }
  __syncthreads();
  return r;
}

// Left move core: C (Dl x 2Dr row-major, in X) = L Q via QR of C^H = Q' R'.
// X <- Q'^H (r, 2, Dr); R' stays in W (column-major, ld 2Dr), L = R'^H.
// Returns r = min(2Dr, Dl). Whole CTA. HR as in qr_right_cta (2 Dr <= 32 HR).
template <typename R, int HR = 0, int NB = sizeof(R) == 4 ? 8 : 4>
__device__ int lq_left_cta(cx<R> *X, int Dl, int Dr, cx<R> *W, cx<R> *Qbuf) {
  const int m = 2 * Dr, n = Dl, r = m < n ? m : n;
  __shared__ cx<R> tau[2 * TNMPS_MAX_CHI];
  __shared__ cx<R> vs[2 * TNMPS_MAX_CHI];
  __shared__ R red[32];
  __syncthreads();
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) W[e] = cconj(X[e]);
  __syncthreads();
  // staged panel + tau/vs arrays within 40 KB of static shared memory
  if constexpr (HR > 0 &&
                (NB * 32 * HR + 4 * TNMPS_MAX_CHI) * sizeof(cx<R>) <= 40960) {
    __shared__ cx<R> Ts[NB * NB], Gs[NB * NB];
    __shared__ __align__(16) cx<R> Vs[NB * 32 * HR];  // the panel's reflectors
    householder_qr_blocked<R, NB, HR>(W, m, n, tau, red, vs, Ts, Gs, Vs);
    householder_form_q_blocked<R, NB, HR>(W, m, n, tau, Qbuf, Ts, Gs, Vs);
  } else {
    householder_qr(W, m, n, tau, red, vs);
    householder_form_q(W, m, n, tau, Qbuf, vs);
  }
  for (int e = threadIdx.x; e < r * m; e += blockDim.x) X[e] = cconj(Qbuf[e]);
  __syncthreads();
  return r;
}

// LQ of a two-site block ahead of its SVD: T (M x N row-major) = L Q^H via
// the QR of T^H = Q R'. Q is not formed: T and L have the same singular values
// and left singular vectors, which is all the split uses (it forms U_k^H T
// from T). Wq (N x M column-major scratch) receives T^H and is factored in
// place; L = R'^H goes column-major (ld M) to Lout: lower trapezoidal, r =
// min(M, N) columns, and columns r..N-1 zero. Returns r. Whole CTA. HR as in
// qr_right_cta (N <= 32 HR).
template <typename R, int HR = 0, int NB = sizeof(R) == 4 ? 8 : 4>
__device__ int lq_theta_cta(const cx<R> *T, int M, int N, cx<R> *Wq, cx<R> *Lout) {
  const int m = N, n = M, r = m < n ? m : n;
  __shared__ cx<R> tau[2 * TNMPS_MAX_CHI];
  __shared__ cx<R> vs[2 * TNMPS_MAX_CHI];
  __shared__ R red[32];
  __syncthreads();
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) Wq[e] = cconj(T[e]);
  __syncthreads();
  if constexpr (HR > 0 &&
                (NB * 32 * HR + 4 * TNMPS_MAX_CHI) * sizeof(cx<R>) <= 40960) {
    __shared__ cx<R> Ts[NB * NB], Gs[NB * NB];
    __shared__ __align__(16) cx<R> Vs[NB * 32 * HR];  // the panel's reflectors
    householder_qr_blocked<R, NB, HR>(Wq, m, n, tau, red, vs, Ts, Gs, Vs);
  } else {
    householder_qr(Wq, m, n, tau, red, vs);
  }
  // L[p][q] = conj(R'[q][p]) for p >= q, q < r; R'[q][p] sits at Wq[q + p m]
  for (int e = threadIdx.x; e < M * N; e += blockDim.x) {
    const int q = e / M, p = e - q * M;
    Lout[e] = (q < r && p >= q) ? cconj(Wq[(int64_t)p * m + q]) : mkc<R>(0, 0);
  }
  __syncthreads();
  return r;
}

}  // namespace gdev
