// Shots of a computational-basis measurement of every qubit -- the MEASURE
// instructions that end the kernels of Sec. V.B -- sampled exactly: qubits
// n-1, ..., 0 in turn, each drawn from its probability conditioned on the
// outcomes already drawn.
//
// Precondition: orthogonality centre on site n-1 (the entry point moves it),
// so sites 0..n-2 are left isometries and
//     P(s | outcomes above q) = ||X_q[:, s, :] v||^2 / (p0 + p1)
// for the normalised conditional vector v of the shot (v = 1 above site n-1).
// The random numbers are inputs: u[b][k][q] decides qubit q of shot k of
// state b, outcome 0 iff u < p0 / (p0 + p1), with p0, p1 accumulated in FP64.
//
// One CTA per (chunk of SC shots, state). The conditional vectors V (D x SC)
// and W_s = X_q[:, s, :] V (2D x SC) live in shared memory; each thread
// computes four outputs of W at a time from one row of X.
#include "tnmps_internal.h"

namespace {

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R, int SC>
__global__ void __launch_bounds__(256) k_sample(StateView sv, const double *__restrict__ u,
                                                int shots, uint8_t *__restrict__ bits,
                                                uint32_t *err) {
  static_assert(SC % 4 == 0 && SC <= 32, "shot chunk");
  const int b = blockIdx.y, k0 = blockIdx.x * SC;
  const int n = sv.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *V = reinterpret_cast<cx<R> *>(smraw);   // [chi][SC]
  cx<R> *W = V + (int64_t)sv.chi * SC;          // [2 chi][SC], row a*2 + s
  __shared__ double p[2][SC];
  __shared__ R scl[SC];
  __shared__ int pick[SC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < SC; e += blockDim.x) V[e] = mkc<R>(1, 0);  // D_{n-1} = 1
  __syncthreads();
  const int32_t *dims = sv.dims + (int64_t)b * (n + 1);
  for (int q = n - 1; q >= 0; --q) {
    const int Dl = dims[q], Dr = dims[q + 1];
    const cx<R> *X = reinterpret_cast<const cx<R> *>(sv.sites) + (int64_t)b * sv.state_elems +
                     sv.site_off[q];
    // W[r][k..k+3] = sum_c X[r][c] V[c][k..k+3], r = (a, s) row of X
    for (int e = threadIdx.x; e < 2 * Dl * (SC / 4); e += blockDim.x) {
      const int k = (e % (SC / 4)) * 4, r = e / (SC / 4);
      cx<R> acc[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = mkc<R>(0, 0);
      const cx<R> *xr = X + (int64_t)r * Dr;
      for (int c = 0; c < Dr; ++c) {
        const cx<R> x = xr[c];
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[j], x, V[c * SC + k + j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) W[r * SC + k + j] = acc[j];
    }
    __syncthreads();
    // p_s[k] = sum_a |W[a*2+s][k]|^2 in FP64
    for (int sk = warp; sk < 2 * SC; sk += nw) {
      const int s = sk / SC, k = sk - s * SC;
      double acc = 0;
      for (int a = lane; a < Dl; a += 32) {
        const cx<R> z = W[(a * 2 + s) * SC + k];
        acc += (double)z.re * z.re + (double)z.im * z.im;
      }
      acc = warp_sum(acc);
      if (lane == 0) p[s][k] = acc;
    }
    __syncthreads();
    if (threadIdx.x < SC) {
      const int k = threadIdx.x;
      int s = 0;
      R sc = 0;
      if (k0 + k < shots) {
        const double p0 = p[0][k], p1 = p[1][k], tot = p0 + p1;
        const double pz = tot > 0 ? p0 / tot : 1.0;
        const int64_t at = ((int64_t)b * shots + k0 + k) * n + q;
        s = u[at] < pz ? 0 : 1;
        const double ps = s ? p1 : p0;
        if (ps > 0 && isfinite(tot)) sc = (R)(1.0 / sqrt(ps));
        else atomicOr(err, TNMPS_EFLAG_NUMERIC);
        bits[at] = (uint8_t)s;
      }
      pick[k] = s;
      scl[k] = sc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Dl * SC; e += blockDim.x) {
      const int k = e % SC, a = e / SC;
      const cx<R> z = W[(a * 2 + pick[k]) * SC + k];
      V[a * SC + k] = mkc<R>(z.re * scl[k], z.im * scl[k]);
    }
    __syncthreads();
  }
}

template <typename R, int SC>
cudaError_t run_sample(tnmps_ctx *c, const double *u, int shots, uint8_t *bits) {
  const size_t smem = (size_t)3 * c->chi * SC * sizeof(cx<R>);
  cudaError_t e = cudaFuncSetAttribute(k_sample<R, SC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((shots + SC - 1) / SC, c->batch);
  k_sample<R, SC><<<grid, 256, smem, c->stream>>>(c->view(), u, shots, bits, c->err);
  ++c->launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sample(tnmps_ctx *c, const double *u, int shots, uint8_t *bits) {
  if (c->dtype == TNMPS_C128) return run_sample<double, 16>(c, u, shots, bits);
  return run_sample<float, 32>(c, u, shots, bits);
}
