// K3: batched one-sided (Hestenes) Jacobi SVD -- the SVD of the two-site
// block that the paper uses to return a rank-4 tensor to MPS form (Sec. II,
// Fig. "mpssvd"; Sec. IV).
//
// Design (GB300): one CTA per matrix (= per state of the batch). The matrix
// stays in global memory (L2-resident for the active CTAs); columns are
// processed in blocks of BC that are staged in shared memory, two blocks at a
// time. Within a staged pair of blocks every column pair is orthogonalised by
// one warp: the warp holds both columns in registers (E elements per lane),
// forms the 2x2 Gram entries alpha = |x|^2, beta = |y|^2, gamma = x^H y with
// a warp reduction and applies the complex rotation that zeroes gamma.
// Concurrent warps work on disjoint column pairs (round-robin ordering inside
// a block, cyclic shifts across two blocks), so a sweep visits every pair of
// columns exactly once. A sweep with no rotation (all pairs within the
// relative tolerance |gamma| <= tol * sqrt(alpha beta)) ends the iteration;
// the sweep cap sets an error flag instead of spinning.
//
// On exit the columns of W are A V with V unitary: mutually orthogonal, with
// norms equal to the singular values. The left singular vectors are the
// normalised columns; the split step recovers Sigma V^H as U^H Theta, so V is
// never accumulated.
#include "tnmps_internal.h"

namespace {

struct JacobiArgs {
  void *W;
  int64_t stride;          // elements between matrices
  const int32_t *dims;     // gate mode: M = 2 dims[b][l], N = 2 dims[b][l+2]
  int dstride, l;
  int m, n, lda;           // fixed mode (dims == nullptr)
  double *sigma_out;       // optional [batch][n]
  int32_t *sweeps_out;     // optional [batch]
  int max_sweeps;
  float tolfac;
  uint32_t *err;
  unsigned long long *counters;
};

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
template <typename R, int E, int NP>
__device__ __forceinline__ int rotate_pairs(cx<R> *const *xs, cx<R> *const *ys, int M, int lane,
                                            R tol2, R tiny) {
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

template <typename R>
__device__ __forceinline__ void load_block(cx<R> *__restrict__ S, const cx<R> *__restrict__ W,
                                           int col0, int ncol, int M, int ld, int Mp) {
  for (int e = threadIdx.x; e < ncol * M; e += blockDim.x) {
    const int c = e / M, r = e - c * M;
    S[c * Mp + r] = W[(int64_t)(col0 + c) * ld + r];
  }
}
template <typename R>
__device__ __forceinline__ void store_block(const cx<R> *__restrict__ S, cx<R> *__restrict__ W,
                                            int col0, int ncol, int M, int ld, int Mp) {
  for (int e = threadIdx.x; e < ncol * M; e += blockDim.x) {
    const int c = e / M, r = e - c * M;
    W[(int64_t)(col0 + c) * ld + r] = S[c * Mp + r];
  }
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
                                        R tiny, int &checked) {
  checked += np;
  int mask = 0;
  if constexpr (TwoPairs<R, E>::ok) {
    if (np == 2) mask = rotate_pairs<R, E, 2>(xs, ys, M, lane, tol2, tiny);
    else if (np == 1) mask = rotate_pairs<R, E, 1>(xs, ys, M, lane, tol2, tiny);
  } else {
    if (np >= 1) mask = rotate_pairs<R, E, 1>(xs, ys, M, lane, tol2, tiny);
    if (np == 2) mask |= rotate_pairs<R, E, 1>(xs + 1, ys + 1, M, lane, tol2, tiny) << 1;
  }
  return (mask & 1) + (mask >> 1);
}

// all pairs inside one staged block (round-robin / circle ordering)
template <typename R, int E>
__device__ int within_block(cx<R> *S, int nc, int M, int Mp, R tol2, R tiny, int &checked) {
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
      rot += do_pairs<R, E>(xs, ys, (int)ok[0] + (int)ok[1], M, lane, tol2, tiny, checked);
    }
    __syncthreads();
  }
  return rot;
}

// all cross pairs between two staged blocks (cyclic shifts)
template <typename R, int E, int BC>
__device__ int cross_blocks(cx<R> *S0, int n0, cx<R> *S1, int n1, int M, int Mp, R tol2, R tiny,
                            int &checked) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int rot = 0;
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
      rot += do_pairs<R, E>(xs, ys, (int)ok[0] + (int)ok[1], M, lane, tol2, tiny, checked);
    }
    __syncthreads();
  }
  return rot;
}

template <typename R, int BC, int E>
__global__ void __launch_bounds__(BC >= 16 ? 512 : 256) k_jacobi(JacobiArgs p) {
  const int b = blockIdx.x;
  int M, N, ld;
  if (p.dims) {
    M = 2 * p.dims[(int64_t)b * p.dstride + p.l];
    N = 2 * p.dims[(int64_t)b * p.dstride + p.l + 2];
    ld = M;
  } else {
    M = p.m;
    N = p.n;
    ld = p.lda;
  }
  constexpr int Mp = 32 * E;
  cx<R> *W = reinterpret_cast<cx<R> *>(p.W) + (int64_t)b * p.stride;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *S[2];
  S[0] = reinterpret_cast<cx<R> *>(smraw);
  S[1] = S[0] + BC * Mp;
  __shared__ int s_rot;

  // relative orthogonality threshold; the constant term covers the warp
  // reduction's rounding, which does not shrink with M
  const R tol = R(p.tolfac) * (sqrt(R(M)) + R(16)) * Eps<R>::u();
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
  int held[2] = {-1, -1};

  auto ensure = [&](int slot, int blk) {
    if (held[slot] == blk) return;
    if (held[slot] >= 0) {
      const int h = held[slot];
      store_block(S[slot], W, h * BC, min(BC, N - h * BC), M, ld, Mp);
    }
    __syncthreads();
    load_block(S[slot], W, blk * BC, min(BC, N - blk * BC), M, ld, Mp);
    held[slot] = blk;
    __syncthreads();
  };

  int sweep = 0, total_rot = 0, checked = 0;  // checked: pairs this warp examined
  bool converged = false;
  while (sweep < p.max_sweeps) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    int rot = 0;
    for (int I = 0; I < nb; ++I) {
      // keep block I in whichever slot already holds it
      int sI = (held[1] == I) ? 1 : 0;
      ensure(sI, I);
      const int nI = min(BC, N - I * BC);
      rot += within_block<R, E>(S[sI], nI, M, Mp, tol2, tiny, checked);
      for (int J = I + 1; J < nb; ++J) {
        ensure(1 - sI, J);
        const int nJ = min(BC, N - J * BC);
        rot += cross_blocks<R, E, BC>(S[sI], nI, S[1 - sI], nJ, M, Mp, tol2, tiny, checked);
      }
    }
    if (rot && (threadIdx.x & 31) == 0) atomicAdd(&s_rot, rot);
    __syncthreads();
    ++sweep;
    const int swept = s_rot;
    __syncthreads();
    total_rot += swept;
    if (swept == 0) {
      converged = true;
      break;
    }
  }
  for (int s = 0; s < 2; ++s)
    if (held[s] >= 0) store_block(S[s], W, held[s] * BC, min(BC, N - held[s] * BC), M, ld, Mp);
  __syncthreads();

  if (p.sigma_out) {  // column norms in FP64
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < N; j += nw) {
      double acc = 0;
      for (int r = lane; r < M; r += 32) {
        const cx<R> z = W[(int64_t)j * ld + r];
        acc += (double)z.re * z.re + (double)z.im * z.im;
      }
      acc = warp_sum(acc);
      if (lane == 0) p.sigma_out[(int64_t)b * N + j] = sqrt(acc);
    }
  }
  if (p.counters && (threadIdx.x & 31) == 0 && checked)
    atomicAdd(&p.counters[CNT_PAIR_ROWS], (unsigned long long)checked * M);
  if (threadIdx.x == 0) {
    if (p.sweeps_out) p.sweeps_out[b] = sweep;
    if (!converged && N > 1 && p.err) atomicOr(p.err, TNMPS_EFLAG_NOT_CONVERGED);
    if (p.counters) {
      atomicAdd(&p.counters[CNT_ROTATIONS], (unsigned long long)total_rot);
      atomicAdd(&p.counters[CNT_ROT_ROWS], (unsigned long long)total_rot * M);
      atomicAdd(&p.counters[CNT_SWEEPS], (unsigned long long)sweep);
      atomicAdd(&p.counters[CNT_SVDS], 1ull);
    }
  }
}

template <typename R, int BC, int E>
cudaError_t run(const JacobiArgs &a, int batch, cudaStream_t s) {
  constexpr int NT = BC >= 16 ? 512 : 256;
  const size_t smem = (size_t)2 * BC * 32 * E * sizeof(cx<R>);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi<R, BC, E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi<R, BC, E><<<batch, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t dispatch(const JacobiArgs &a, int Mcap, int batch, cudaStream_t s) {
  if (Mcap <= 64) return run<R, 32, 2>(a, batch, s);
  if (Mcap <= 128) return run<R, 32, 4>(a, batch, s);
  if (Mcap <= 256) return run<R, sizeof(R) == 8 ? 16 : 32, 8>(a, batch, s);
  return run<R, sizeof(R) == 8 ? 8 : 16, 16>(a, batch, s);
}

}  // namespace

// gate mode: matrix of state b is the W buffer, M = 2 D_{l-1}, N = 2 D_{l+1}
cudaError_t launch_jacobi_gate(tnmps_ctx *c, int l, int Mcap) {
  JacobiArgs a{};
  a.W = c->w_buf;
  a.stride = c->tw;
  a.dims = c->dims;
  a.dstride = c->n + 1;
  a.l = l;
  a.max_sweeps = c->dtype == TNMPS_C128 ? 40 : 30;
  a.tolfac = 1.0f;
  a.err = c->err;
  a.counters = c->counters;
  if (c->dtype == TNMPS_C128) return dispatch<double>(a, Mcap, c->batch, c->stream);
  return dispatch<float>(a, Mcap, c->batch, c->stream);
}

cudaError_t launch_jacobi_standalone(tnmps_dtype dt, int batch, int m, int n, void *A, int lda,
                                     double *sigma, int32_t *sweeps, int max_sweeps,
                                     cudaStream_t s) {
  JacobiArgs a{};
  a.W = A;
  a.stride = (int64_t)lda * n;
  a.m = m;
  a.n = n;
  a.lda = lda;
  a.sigma_out = sigma;
  a.sweeps_out = sweeps;
  a.max_sweeps = max_sweeps > 0 ? max_sweeps : (dt == TNMPS_C128 ? 40 : 30);
  a.tolfac = 1.0f;
  if (dt == TNMPS_C128) return dispatch<double>(a, m, batch, s);
  return dispatch<float>(a, m, batch, s);
}
