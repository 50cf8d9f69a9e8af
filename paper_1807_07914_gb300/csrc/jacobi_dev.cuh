// Device building blocks of the one-sided Jacobi SVD (shared by the batched
// gate-step kernel and the persistent multi-circuit kernel).
#pragma once
#include "tnmps_internal.h"

namespace jac {


template <typename R>
struct Eps;
template <>
struct Eps<double> {
  static __device__ __forceinline__ double u() { return 1.1102230246251565e-16; }
};
template <>
struct Eps<float> {
  static __device__ __forceinline__ float u() { return 5.9604645e-08f; }
};

// scalar helpers: hardware approximations in FP32 (the rotation only has to
// be orthogonal to a few ulp; the split re-orthonormalises), IEEE in FP64
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double frsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lane-to-element map of a column held in registers: with V complex values
// per 16-byte vector (V = 2 for complex64, 1 for complex128), register e of
// a lane holds element (e / V) * 32V + lane * V + e % V, so a warp reads a
// column with conflict-free 16-byte shared-memory accesses.
template <typename R>
struct Vec;
template <>
struct Vec<float> {
  static constexpr int V = 2;
  __device__ static __forceinline__ void ld(const cx<float> *p, cx<float> &a, cx<float> &b) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    a = mkc<float>(q.x, q.y);
    b = mkc<float>(q.z, q.w);
  }
  __device__ static __forceinline__ void st(cx<float> *p, cx<float> a, cx<float> b) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.re, a.im, b.re, b.im);
  }
};
template <>
struct Vec<double> {
  static constexpr int V = 1;
};

template <typename R, int E>
__device__ __forceinline__ void load_col(const cx<R> *__restrict__ x, int M, int lane, cx<R> *v) {
  constexpr int V = Vec<R>::V;
#pragma unroll
  for (int j = 0; j < E / V; ++j) {
    const int r = j * 32 * V + lane * V;
    if constexpr (V == 2) {
      if (r < M) Vec<R>::ld(x + r, v[2 * j], v[2 * j + 1]);   // M is even
      else v[2 * j] = v[2 * j + 1] = mkc<R>(0, 0);
    } else {
      v[j] = r < M ? x[r] : mkc<R>(0, 0);
    }
  }
}
template <typename R, int E>
__device__ __forceinline__ void store_col(cx<R> *__restrict__ x, int M, int lane, const cx<R> *v) {
  constexpr int V = Vec<R>::V;
#pragma unroll
  for (int j = 0; j < E / V; ++j) {
    const int r = j * 32 * V + lane * V;
    if (r < M) {
      if constexpr (V == 2) Vec<R>::st(x + r, v[2 * j], v[2 * j + 1]);
      else x[r] = v[j];
    }
  }
}

// Sum K = 4 NP per-lane partial sums over the warp: halving exchanges leave
// value j in lane (32 / K) * j, which then broadcasts it.
template <typename R, int K>
__device__ __forceinline__ void warp_reduce_all(R *v, int lane) {
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

// Orthogonalise NP column pairs (x[p], y[p]) of length M in shared memory
// at once (independent pairs interleave their latency chains). Returns a
// bitmask of the pairs rotated.
// dmax2: running maximum of |gamma|^2 / (alpha beta) over the pairs rotated.
template <typename R, int E, int NP>
__device__ __forceinline__ int rotate_pairs(cx<R> *const *xs, cx<R> *const *ys, int M, int lane,
                                            R tol2, R tiny, R &dmax2) {
  cx<R> xv[NP][E], yv[NP][E];
  R acc[4 * NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    load_col<R, E>(xs[p], M, lane, xv[p]);
    load_col<R, E>(ys[p], M, lane, yv[p]);
    R a = 0, bb = 0, gr = 0, gi = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      a = fma(xv[p][e].re, xv[p][e].re, fma(xv[p][e].im, xv[p][e].im, a));
      bb = fma(yv[p][e].re, yv[p][e].re, fma(yv[p][e].im, yv[p][e].im, bb));
      gr = fma(xv[p][e].re, yv[p][e].re, fma(xv[p][e].im, yv[p][e].im, gr));   // Re(conj(x) y)
      gi = fma(xv[p][e].re, yv[p][e].im, fma(-xv[p][e].im, yv[p][e].re, gi));  // Im(conj(x) y)
    }
    acc[4 * p] = a;
    acc[4 * p + 1] = bb;
    acc[4 * p + 2] = gr;
    acc[4 * p + 3] = gi;
  }
  warp_reduce_all<R, 4 * NP>(acc, lane);
  int rotated = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const R a = acc[4 * p], bb = acc[4 * p + 1], gr = acc[4 * p + 2], gi = acc[4 * p + 3];
    // columns at the rounding-noise floor are left alone: they cannot be made
    // relatively orthogonal (there may be no room for them) and the split
    // always truncates them
    if (!(a > tiny && bb > tiny)) continue;
    const R g2 = gr * gr + gi * gi;
    if (!(g2 > tol2 * a * bb)) continue;
    dmax2 = fmax(dmax2, g2 / (a * bb));
    // real Jacobi rotation on (x, e^{-i phi} y), gamma = g e^{i phi}
    const R ig = frsqrt(g2);  // 1 / |gamma|
    const R zeta = (bb - a) * (R(0.5) * ig);
    const R t = copysign(R(1), zeta) * frcp(fabs(zeta) + (R(1) + zeta * zeta) * frsqrt(R(1) + zeta * zeta));
    const R c = frsqrt(R(1) + t * t);
    const R s = c * t;
    const R er = gr * ig, ei = -gi * ig;  // e^{-i phi}
    const R ser = s * er, sei = s * ei, cer = c * er, cei = c * ei;
    // x' = c x - s e y,  y' = s x + c e y
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const cx<R> x = xv[p][e], y = yv[p][e];
      xv[p][e] = mkc<R>(fma(c, x.re, fma(-ser, y.re, sei * y.im)),
                        fma(c, x.im, fma(-ser, y.im, -sei * y.re)));
      yv[p][e] = mkc<R>(fma(s, x.re, fma(cer, y.re, -cei * y.im)),
                        fma(s, x.im, fma(cer, y.im, cei * y.re)));
    }
    store_col<R, E>(xs[p], M, lane, xv[p]);
    store_col<R, E>(ys[p], M, lane, yv[p]);
    rotated |= 1 << p;
  }
  return rotated;
}

// Block staging between the matrix in global memory (L2) and shared memory:
// a warp per column, 16-byte vectors with all of a lane's loads in flight
// together; element-wise when the column starts are not 16-byte aligned.
template <typename R>
__device__ __forceinline__ bool vec_ok(const cx<R> *W, int M, int ld) {
  constexpr int V = sizeof(cx<R>) == 8 ? 2 : 1;  // complex values per 16 bytes
  return (reinterpret_cast<uintptr_t>(W) & 15) == 0 && (M % V) == 0 && (ld % V) == 0;
}

// Block slot c holds matrix column perm[col0 + c].
template <typename R>
__device__ __forceinline__ void load_block(cx<R> *__restrict__ S, const cx<R> *__restrict__ W,
                                           const int *perm, int col0, int ncol, int M, int ld,
                                           int Mp) {
  if (vec_ok(W, M, ld)) {
    constexpr int V = sizeof(cx<R>) == 8 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nv = M / V;
    for (int c = warp; c < ncol; c += nw) {
      const float4 *src = reinterpret_cast<const float4 *>(W + (int64_t)perm[col0 + c] * ld);
      float4 *dst = reinterpret_cast<float4 *>(S + c * Mp);
#pragma unroll 4
      for (int v = lane; v < nv; v += 32) dst[v] = src[v];
    }
    return;
  }
  for (int e = threadIdx.x; e < ncol * M; e += blockDim.x) {
    const int c = e / M, r = e - c * M;
    S[c * Mp + r] = W[(int64_t)perm[col0 + c] * ld + r];
  }
}
template <typename R>
__device__ __forceinline__ void store_block(const cx<R> *__restrict__ S, cx<R> *__restrict__ W,
                                            const int *perm, int col0, int ncol, int M, int ld,
                                            int Mp) {
  if (vec_ok(W, M, ld)) {
    constexpr int V = sizeof(cx<R>) == 8 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nv = M / V;
    for (int c = warp; c < ncol; c += nw) {
      const float4 *src = reinterpret_cast<const float4 *>(S + c * Mp);
      float4 *dst = reinterpret_cast<float4 *>(W + (int64_t)perm[col0 + c] * ld);
#pragma unroll 4
      for (int v = lane; v < nv; v += 32) dst[v] = src[v];
    }
    return;
  }
  for (int e = threadIdx.x; e < ncol * M; e += blockDim.x) {
    const int c = e / M, r = e - c * M;
    W[(int64_t)perm[col0 + c] * ld + r] = S[c * Mp + r];
  }
}

// Asynchronous 16-byte global -> shared copies (cp.async, generic proxy);
// cp_async_wait_all completes the calling thread's copies.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// load_block issued as asynchronous copies, with the thread <-> element map
// of store_block (a thread overwrites only what it wrote back itself, so a
// store_block / prefetch_block pair on one slot needs no barrier between).
// The element-wise path (unaligned columns) copies synchronously.
template <typename R>
__device__ __forceinline__ void prefetch_block(cx<R> *__restrict__ S,
                                               const cx<R> *__restrict__ W, const int *perm,
                                               int col0, int ncol, int M, int ld, int Mp) {
  if (vec_ok(W, M, ld)) {
    constexpr int V = sizeof(cx<R>) == 8 ? 2 : 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nv = M / V;
    for (int c = warp; c < ncol; c += nw) {
      const float4 *src = reinterpret_cast<const float4 *>(W + (int64_t)perm[col0 + c] * ld);
      float4 *dst = reinterpret_cast<float4 *>(S + c * Mp);
      for (int v = lane; v < nv; v += 32) cp_async16(dst + v, src + v);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    return;
  }
  load_block(S, W, perm, col0, ncol, M, ld, Mp);
}

// A warp's share of one round: up to two disjoint pairs, processed together.
// Two pairs at once only while both fit in registers (8E floats or 16E
// doubles of column data per lane).
template <typename R, int E>
struct TwoPairs {
  static constexpr bool ok = sizeof(R) == 4 ? E <= 8 : E <= 4;
};

// A warp's share of one round: up to two disjoint pairs, processed together
// (compile-time indices only, so the pointers stay in registers).
template <typename R, int E>
__device__ __forceinline__ int do_pairs(cx<R> **xs, cx<R> **ys, int np, int M, int lane, R tol2,
                                        R tiny, int &checked, R &dmax2) {
  checked += np;
  int mask = 0;
  if constexpr (TwoPairs<R, E>::ok) {
    if (np == 2) mask = rotate_pairs<R, E, 2>(xs, ys, M, lane, tol2, tiny, dmax2);
    else if (np == 1) mask = rotate_pairs<R, E, 1>(xs, ys, M, lane, tol2, tiny, dmax2);
  } else {
    if (np >= 1) mask = rotate_pairs<R, E, 1>(xs, ys, M, lane, tol2, tiny, dmax2);
    if (np == 2) mask |= rotate_pairs<R, E, 1>(xs + 1, ys + 1, M, lane, tol2, tiny, dmax2) << 1;
  }
  return (mask & 1) + (mask >> 1);
}

// all pairs inside one staged block (round-robin / circle ordering)
template <typename R, int E>
__device__ int within_block(cx<R> *S, int nc, int M, int Mp, R tol2, R tiny, int &checked,
                            R &dmax2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int rot = 0;
  if (nc < 2) return 0;
  const int m = (nc + 1) & ~1;
  for (int r = 0; r < m - 1; ++r) {
    for (int k0 = warp; k0 < m / 2; k0 += 2 * nw) {
      cx<R> *xs[2], *ys[2];
      bool ok[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = k0 + q * nw;
        const int a = (r + k) % (m - 1);
        const int b = (k == 0) ? (m - 1) : (r - k + (m - 1)) % (m - 1);
        ok[q] = k < m / 2 && a < nc && b < nc;
        xs[q] = S + a * Mp;
        ys[q] = S + b * Mp;
      }
      if (!ok[0] && ok[1]) {
        xs[0] = xs[1];
        ys[0] = ys[1];
      }
      rot += do_pairs<R, E>(xs, ys, (int)ok[0] + (int)ok[1], M, lane, tol2, tiny, checked, dmax2);
    }
    __syncthreads();
  }
  return rot;
}

// One y column (shared memory) against the warp's two register-resident x
// columns in turn: pair A = (x1, y), then pair B = (x2, y'), y' = y after A.
// All dot products are formed before either rotation (one warp reduction):
// alpha1, beta, gamma1 = x1^H y, alpha2, h = x2^H y, q = x2^H x1; then
// gamma_B = x2^H y' = s1 q + c1 e1 h and beta' = beta + t1 |gamma1| exactly.
// valid[]: x1 / x2 / y present. Returns the number of rotations.
// ax[] carries |x1|^2, |x2|^2 through the rounds (the x columns only change
// here): alpha - t |gamma| after a rotation, recomputed from the registers
// when that update cancels by more than 100x.
template <typename R, int E>
__device__ __forceinline__ R col_norm2(const cx<R> (&v)[E]) {
  R q = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) q = fma(v[e].re, v[e].re, fma(v[e].im, v[e].im, q));
  return warp_sum(q);
}

template <typename R, int E>
__device__ __forceinline__ int rotate_x2y(cx<R> (&xv)[2][E], R (&ax)[2], cx<R> *ys,
                                          const bool *valid, int M, int lane, R tol2, R tiny,
                                          R &dmax2) {
  cx<R> yv[E];
  if (valid[2]) load_col<R, E>(ys, M, lane, yv);
  else
#pragma unroll
    for (int e = 0; e < E; ++e) yv[e] = mkc<R>(0, 0);
  R acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const cx<R> x1 = xv[0][e], x2 = xv[1][e], y = yv[e];
    acc[1] = fma(y.re, y.re, fma(y.im, y.im, acc[1]));       // beta
    acc[2] = fma(x1.re, y.re, fma(x1.im, y.im, acc[2]));     // Re x1^H y
    acc[3] = fma(x1.re, y.im, fma(-x1.im, y.re, acc[3]));    // Im x1^H y
    acc[4] = fma(x2.re, y.re, fma(x2.im, y.im, acc[4]));     // Re x2^H y
    acc[5] = fma(x2.re, y.im, fma(-x2.im, y.re, acc[5]));    // Im x2^H y
    acc[6] = fma(x2.re, x1.re, fma(x2.im, x1.im, acc[6]));   // Re x2^H x1
    acc[7] = fma(x2.re, x1.im, fma(-x2.im, x1.re, acc[7]));  // Im x2^H x1
  }
  warp_reduce_all<R, 8>(acc, lane);
  acc[0] = ax[0];
  const R a2 = ax[1];
  int rotated = 0;
  R beta = acc[1], gr = acc[4], gi = acc[5];  // pair B's beta and gamma if A does not rotate
  // pair A
  if (valid[0] && valid[2] && acc[0] > tiny && beta > tiny) {
    const R g1r = acc[2], g1i = acc[3], g2 = g1r * g1r + g1i * g1i;
    if (g2 > tol2 * acc[0] * beta) {
      dmax2 = fmax(dmax2, g2 / (acc[0] * beta));
      const R ig = frsqrt(g2);
      const R zeta = (beta - acc[0]) * (R(0.5) * ig);
      const R t = copysign(R(1), zeta) * frcp(fabs(zeta) + (R(1) + zeta * zeta) * frsqrt(R(1) + zeta * zeta));
      const R c = frsqrt(R(1) + t * t);
      const R s = c * t;
      const R er = g1r * ig, ei = -g1i * ig;  // e^{-i phi}
      const R ser = s * er, sei = s * ei, cer = c * er, cei = c * ei;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const cx<R> x = xv[0][e], y = yv[e];
        xv[0][e] = mkc<R>(fma(c, x.re, fma(-ser, y.re, sei * y.im)),
                          fma(c, x.im, fma(-ser, y.im, -sei * y.re)));
        yv[e] = mkc<R>(fma(s, x.re, fma(cer, y.re, -cei * y.im)),
                       fma(s, x.im, fma(cer, y.im, cei * y.re)));
      }
      const R tg = t * (g2 * ig);  // t |gamma|
      beta = beta + tg;
      ax[0] = acc[0] - tg;
      if (!(ax[0] > R(0.01) * acc[0])) ax[0] = col_norm2<R, E>(xv[0]);
      // x2^H y' = s q + c e h
      gr = fma(s, acc[6], fma(cer, acc[4], -cei * acc[5]));
      gi = fma(s, acc[7], fma(cer, acc[5], cei * acc[4]));
      ++rotated;
    }
  }
  // pair B on y'
  if (valid[1] && valid[2] && a2 > tiny && beta > tiny) {
    const R g2 = gr * gr + gi * gi;
    if (g2 > tol2 * a2 * beta) {
      dmax2 = fmax(dmax2, g2 / (a2 * beta));
      const R ig = frsqrt(g2);
      const R zeta = (beta - a2) * (R(0.5) * ig);
      const R t = copysign(R(1), zeta) * frcp(fabs(zeta) + (R(1) + zeta * zeta) * frsqrt(R(1) + zeta * zeta));
      const R c = frsqrt(R(1) + t * t);
      const R s = c * t;
      const R er = gr * ig, ei = -gi * ig;
      const R ser = s * er, sei = s * ei, cer = c * er, cei = c * ei;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const cx<R> x = xv[1][e], y = yv[e];
        xv[1][e] = mkc<R>(fma(c, x.re, fma(-ser, y.re, sei * y.im)),
                          fma(c, x.im, fma(-ser, y.im, -sei * y.re)));
        yv[e] = mkc<R>(fma(s, x.re, fma(cer, y.re, -cei * y.im)),
                       fma(s, x.im, fma(cer, y.im, cei * y.re)));
      }
      ax[1] = a2 - t * (g2 * ig);
      if (!(ax[1] > R(0.01) * a2)) ax[1] = col_norm2<R, E>(xv[1]);
      ++rotated;
    }
  }
  if (rotated) store_col<R, E>(ys, M, lane, yv);
  return rotated;
}

// all cross pairs between two staged blocks (cyclic shifts). XREG (a CTA of
// BC / 2 warps): warp w owns S0 columns w and w + BC/2 for all rounds and
// keeps them in registers, and each round passes one S1 column through both,
// so only one column per two pairs moves through shared memory.
template <typename R, int E, int BC, bool XREG = false>
__device__ int cross_blocks(cx<R> *S0, int n0, cx<R> *S1, int n1, int M, int Mp, R tol2, R tiny,
                            int &checked, R &dmax2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int rot = 0;
  if constexpr (XREG) {
    static_assert(TwoPairs<R, E>::ok, "two register-resident pairs per warp");
    {
      cx<R> xv[2][E];
      R ax[2];
      const bool have[2] = {warp < n0, warp + nw < n0};
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (have[q]) load_col<R, E>(S0 + (warp + q * nw) * Mp, M, lane, xv[q]);
        else
#pragma unroll
          for (int e = 0; e < E; ++e) xv[q][e] = mkc<R>(0, 0);
        ax[q] = col_norm2<R, E>(xv[q]);
      }
      // round t: warp w takes S1 column (w + t) % BC through its x columns
      // w and w + nw in turn -- every (S0, S1) pair once over the BC rounds
      for (int t = 0; t < BC; ++t) {
        const int j = (warp + t) % BC;
        const bool valid[3] = {have[0], have[1], j < n1};
        checked += valid[2] ? (int)have[0] + (int)have[1] : 0;
        rot += rotate_x2y<R, E>(xv, ax, S1 + j * Mp, valid, M, lane, tol2, tiny, dmax2);
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 2; ++q)
        if (have[q]) store_col<R, E>(S0 + (warp + q * nw) * Mp, M, lane, xv[q]);
      __syncthreads();
      return rot;
    }
  } else {
  for (int t = 0; t < BC; ++t) {
    for (int k0 = warp; k0 < BC; k0 += 2 * nw) {
      cx<R> *xs[2], *ys[2];
      bool ok[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int k = k0 + q * nw;
        const int j = (k + t) % BC;
        ok[q] = k < BC && k < n0 && j < n1;
        xs[q] = S0 + k * Mp;
        ys[q] = S1 + j * Mp;
      }
      if (!ok[0] && ok[1]) {
        xs[0] = xs[1];
        ys[0] = ys[1];
      }
      rot += do_pairs<R, E>(xs, ys, (int)ok[0] + (int)ok[1], M, lane, tol2, tiny, checked, dmax2);
    }
    __syncthreads();
  }
  return rot;
  }
}


// One-sided Jacobi on the column-major M x N matrix W (ld >= M) by the whole
// CTA, columns staged BC at a time in the dynamic shared memory S0/S1 (each
// BC x 32E complex). Returns the number of sweeps run; *converged tells
// whether the last sweep rotated nothing; *rotations / *checked count pair
// visits (per thread: warps add their own). XREG: see cross_blocks (the CTA
// must then have BC / 2 warps).
template <typename R, int BC, int E, bool XREG = false, bool PF = false>
__device__ int jacobi_run(cx<R> *W, int M, int N, int ld, cx<R> *S0, cx<R> *S1, float tolfac,
                          int max_sweeps, bool *converged, int *rotations, int *checked,
                          cx<R> *S2 = nullptr) {
  constexpr int Mp = 32 * E;
  constexpr int NS = PF ? 3 : 2;  // staging slots; PF: the third takes the next block early
  cx<R> *S[3] = {S0, S1, S2};
  __shared__ int s_rot;
  __shared__ unsigned s_dmax;
  const R tol = R(tolfac) * (sqrt(R(M)) + R(16)) * Eps<R>::u();
  const R tol2 = tol * tol;
  // noise floor: (8 u ||A||_F)^2 on squared column norms (||A||_F is invariant)
  __shared__ double s_fro[32];
  {
    double part = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)M * N; e += blockDim.x) {
      const int c = (int)(e / M), r = (int)(e - (int64_t)c * M);
      const cx<R> z = W[(int64_t)c * ld + r];
      part += (double)z.re * z.re + (double)z.im * z.im;
    }
    part = warp_sum(part);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_fro[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_fro[w];
      s_fro[0] = t;
    }
    __syncthreads();
  }
  const R tiny = (R)((64.0 * (double)Eps<R>::u() * (double)Eps<R>::u()) * s_fro[0]);
  const int nb = (N + BC - 1) / BC;
  int held[3] = {-1, -1, -1};
  // column order of the sweep: the blocks are groups of BC consecutive
  // entries of s_perm (matrix columns sorted by descending norm each sweep)
  __shared__ int s_perm[TNMPS_JACOBI_MAX_DIM];
  __shared__ float s_key[TNMPS_JACOBI_MAX_DIM];
  for (int c = threadIdx.x; c < N; c += blockDim.x) s_perm[c] = c;
  __syncthreads();

  auto ensure = [&](int slot, int blk) {
    if (held[slot] == blk) return;
    if (held[slot] >= 0) {
      const int h = held[slot];
      store_block(S[slot], W, s_perm, h * BC, min(BC, N - h * BC), M, ld, Mp);
    }
    __syncthreads();
    load_block(S[slot], W, s_perm, blk * BC, min(BC, N - blk * BC), M, ld, Mp);
    held[slot] = blk;
    __syncthreads();
  };

  int sweep = 0, total_rot = 0, chk = 0;
  bool conv = false;
  while (sweep < max_sweeps) {
    // de Rijk ordering: every sweep visits the columns by descending norm
    // (staged blocks written back first; ties keep the index order)
    for (int s = 0; s < NS; ++s)
      if (held[s] >= 0) {
        store_block(S[s], W, s_perm, held[s] * BC, min(BC, N - held[s] * BC), M, ld, Mp);
        held[s] = -1;
      }
    __syncthreads();
    {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int c = warp; c < N; c += nw) {
        float q = 0;
        for (int r = lane; r < M; r += 32) {
          const cx<R> z = W[(int64_t)c * ld + r];
          q = fmaf((float)z.re, (float)z.re, fmaf((float)z.im, (float)z.im, q));
        }
        q = warp_sum(q);
        if (lane == 0) s_key[c] = q;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float ki = s_key[i];
        int rank = 0;
        for (int j = 0; j < N; ++j) {
          const float kj = s_key[j];
          rank += (kj > ki || (kj == ki && j < i)) ? 1 : 0;
        }
        s_perm[rank] = i;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_dmax = 0u;
    }
    __syncthreads();
    int rot = 0;
    R dmax2 = 0;
    if constexpr (PF) {
      // steps (I, I), (I, I+1), ..., (I, nb-1), (I+1, I+1), ...: each step
      // needs at most one block that is not staged yet, which is copied into
      // the slot neither this step nor the next uses (written back first)
      // while this step computes
      auto slot_of = [&](int blk) {
        for (int s = 0; s < 3; ++s)
          if (held[s] == blk) return s;
        return -1;
      };
      load_block(S[0], W, s_perm, 0, min(BC, N), M, ld, Mp);
      held[0] = 0;
      __syncthreads();
      int I = 0, J = 0;
      for (;;) {
        int nI = I, nJ = J + 1;
        if (nJ >= nb) {
          nI = I + 1;
          nJ = nI;
        }
        const bool more = nI < nb;
        const int sX = slot_of(I), sY = slot_of(J);
        if (more) {
          const int need = slot_of(nI) < 0 ? nI : (slot_of(nJ) < 0 ? nJ : -1);
          if (need >= 0) {
            int t = -1;  // empty slot first, then the lowest block (done for this sweep)
            for (int s = 0; s < 3; ++s) {
              if (s == sX || s == sY || held[s] == nI || held[s] == nJ) continue;
              if (t < 0 || held[s] < held[t]) t = s;
            }
            if (held[t] >= 0)
              store_block(S[t], W, s_perm, held[t] * BC, min(BC, N - held[t] * BC), M, ld, Mp);
            prefetch_block(S[t], W, s_perm, need * BC, min(BC, N - need * BC), M, ld, Mp);
            held[t] = need;
          }
        }
        const int nX = min(BC, N - I * BC);
        if (I == J)
          rot += within_block<R, E>(S[sX], nX, M, Mp, tol2, tiny, chk, dmax2);
        else
          rot += cross_blocks<R, E, BC, XREG>(S[sX], nX, S[sY], min(BC, N - J * BC), M, Mp,
                                              tol2, tiny, chk, dmax2);
        cp_async_wait_all();
        __syncthreads();
        if (!more) break;
        I = nI;
        J = nJ;
      }
    } else {
      for (int I = 0; I < nb; ++I) {
        int sI = (held[1] == I) ? 1 : 0;
        ensure(sI, I);
        const int nI = min(BC, N - I * BC);
        rot += within_block<R, E>(S[sI], nI, M, Mp, tol2, tiny, chk, dmax2);
        for (int J = I + 1; J < nb; ++J) {
          ensure(1 - sI, J);
          const int nJ = min(BC, N - J * BC);
          rot += cross_blocks<R, E, BC, XREG>(S[sI], nI, S[1 - sI], nJ, M, Mp, tol2, tiny, chk,
                                              dmax2);
        }
      }
    }
    if (rot && (threadIdx.x & 31) == 0) {
      atomicAdd(&s_rot, rot);
      atomicMax(&s_dmax, __float_as_uint((float)dmax2));  // non-negative: bits order as values
    }
    __syncthreads();
    ++sweep;
    const int swept = s_rot;
    const float sweep_dmax2 = __uint_as_float(s_dmax);
    __syncthreads();
    total_rot += swept;
    // quadratic convergence: a sweep whose largest relative rotation |gamma| /
    // sqrt(alpha beta) is below sqrt(tol) / 4 leaves every pair within about
    // tol (the next sweep would rotate nothing), so it ends the iteration
    if (swept > 0 && sweep_dmax2 < 0.0625f * (float)tol) {
      conv = true;
      break;
    }
    if (swept == 0) {
      conv = true;
      break;
    }
  }
  for (int s = 0; s < NS; ++s)
    if (held[s] >= 0)
      store_block(S[s], W, s_perm, held[s] * BC, min(BC, N - held[s] * BC), M, ld, Mp);
  __syncthreads();
  *converged = conv;
  *rotations = total_rot;
  *checked = chk;
  return sweep;
}

}  // namespace jac
