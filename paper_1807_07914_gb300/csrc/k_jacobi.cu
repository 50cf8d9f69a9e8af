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

#include "jacobi_dev.cuh"

namespace {

struct JacobiArgs {
  void *W;
  int64_t stride;          // elements between matrices
  const int32_t *dims;     // gate mode: M = 2 dims[b][l], N = 2 dims[b][l+2]
  int dstride, l;
  int n_le_m;              // gate mode: N capped at M (the input is L of Theta = L Q^H)
  int m, n, lda;           // fixed mode (dims == nullptr)
  double *sigma_out;       // optional [batch][n]
  int32_t *sweeps_out;     // optional [batch]
  int max_sweeps;
  float tolfac;
  uint32_t *err;
  unsigned long long *counters;
};

template <typename R, int BC, int E, int NT, int MINB, bool PF>
__global__ void __launch_bounds__(NT, MINB) k_jacobi(JacobiArgs p) {
  const int b = blockIdx.x;
  int M, N, ld;
  if (p.dims) {
    M = 2 * p.dims[(int64_t)b * p.dstride + p.l];
    N = 2 * p.dims[(int64_t)b * p.dstride + p.l + 2];
    if (p.n_le_m && N > M) N = M;  // L has M columns; the rest of the buffer is zero
    ld = M;
  } else {
    M = p.m;
    N = p.n;
    ld = p.lda;
  }
  cx<R> *W = reinterpret_cast<cx<R> *>(p.W) + (int64_t)b * p.stride;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *S0 = reinterpret_cast<cx<R> *>(smraw);
  cx<R> *S1 = S0 + BC * 32 * E;
  cx<R> *S2 = PF ? S1 + BC * 32 * E : nullptr;
  bool converged;
  int total_rot, checked;
  // x columns of the cross rounds in registers when the CTA has BC / 2 warps
  constexpr bool XREG = jac::TwoPairs<R, E>::ok && NT == 16 * BC;
  const int sweep = jac::jacobi_run<R, BC, E, XREG, PF>(W, M, N, ld, S0, S1, p.tolfac,
                                                        p.max_sweeps, &converged, &total_rot,
                                                        &checked, S2);
  if (p.sigma_out) {  // column norms in FP64
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < N; j += nw) {
      double acc = 0;
      for (int r = lane; r < M; r += 32) {
        const cx<R> z = W[(int64_t)j * ld + r];
        acc += (double)z.re * z.re + (double)z.im * z.im;
      }
      acc = jac::warp_sum(acc);
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
      // algorithmic bytes: the matrix read once and written once
      atomicAdd(&p.counters[CNT_JAC_BYTES], 2ull * M * N * sizeof(cx<R>));
    }
  }
}

// NT threads (XREG when NT = 16 BC); MINB CTAs per SM; PF: three staging
// slots, the next block copied asynchronously while the current step computes
template <typename R, int BC, int E, int NT = (BC >= 16 ? 512 : 256), int MINB = 1,
          bool PF = false>
cudaError_t run(const JacobiArgs &a, int batch, cudaStream_t s) {
  const size_t smem = (size_t)(PF ? 3 : 2) * BC * 32 * E * sizeof(cx<R>);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi<R, BC, E, NT, MINB, PF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_jacobi<R, BC, E, NT, MINB, PF><<<batch, NT, smem, s>>>(a);
  return cudaGetLastError();
}

// shape[c] (complex64, blocks of up to 64 / 128 / 256 rows): the launch shape
// chosen by tnmps_set_tuning (0: default, 1: alternative; see tnmps.h)
template <typename R>
cudaError_t dispatch(const JacobiArgs &a, int Mcap, int batch, cudaStream_t s,
                     const int32_t *shape = nullptr) {
  const bool alt0 = sizeof(R) == 4 && shape && shape[0] == 1;
  const bool alt1 = sizeof(R) == 4 && shape && shape[1] == 1;
  const bool alt2 = sizeof(R) == 4 && shape && shape[2] == 1;
  if constexpr (sizeof(R) == 4) {
    if (Mcap <= 64 && alt0) return run<R, 16, 2, 256, 2, true>(a, batch, s);
    if (Mcap > 64 && Mcap <= 128 && alt1) return run<R, 16, 4, 256, 2, true>(a, batch, s);
  }
  if (Mcap <= 64) return run<R, 32, 2, 512, 1, true>(a, batch, s);
  if (Mcap <= 128) return run<R, 32, 4, 512, 1, true>(a, batch, s);
  if constexpr (sizeof(R) == 4) {  // default: 16-column blocks, 8 warps, two CTAs per SM
    if (Mcap <= 256)
      return alt2 ? run<R, 32, 8, 512, 1, true>(a, batch, s)
                  : run<R, 16, 8, 256, 2, true>(a, batch, s);
  }
  if (Mcap <= 256) return run<R, sizeof(R) == 8 ? 16 : 32, 8, 512, 1, true>(a, batch, s);
  return run<R, sizeof(R) == 8 ? 8 : 16, 16, sizeof(R) == 8 ? 256 : 512, 1, true>(a, batch, s);
}

}  // namespace

// gate mode: matrix of state b is the W buffer, M = 2 D_{l-1}, N = 2 D_{l+1}
// (lq: W holds L of Theta = L Q^H, min(M, N) columns)
cudaError_t launch_jacobi_gate(tnmps_ctx *c, int l, int Mcap, bool lq) {
  JacobiArgs a{};
  a.W = c->w_buf;
  a.stride = c->tw;
  a.dims = c->dims;
  a.dstride = c->n + 1;
  a.l = l;
  a.n_le_m = lq ? 1 : 0;
  a.max_sweeps = c->dtype == TNMPS_C128 ? 40 : 30;
  a.tolfac = c->jacobi_tolfac;
  a.err = c->err;
  a.counters = c->counters;
  if (c->dtype == TNMPS_C128) return dispatch<double>(a, Mcap, c->batch, c->stream);
  return dispatch<float>(a, Mcap, c->batch, c->stream, c->tuning.jacobi_shape);
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
