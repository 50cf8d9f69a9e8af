// Gate-step kernels of the MPS update (paper Sec. II Fig. "mpssvd" and Sec. IV):
//   K2  two-site block  Theta[(a,s1),(s2,b)] = sum G[s1 s2, s1' s2'] (C_l B_{l+1})[(a,s1'),(s2',b)]
//   K4  truncate + split: sigma, rank by the cutoff rule, A_l <- U_k,
//       C_{l+1} <- U_k^H Theta / ||sigma_kept||
//   K1  standalone single-qubit gate on a site tensor
//   K7  gauge moves of the orthogonality centre (Householder QR / LQ)
//
// Gauge: mixed canonical form. A two-qubit gate on (l, l+1) is applied with
// the centre on l; afterwards A_l is a left isometry (columns of U) and the
// centre C_{l+1} = Sigma_k V_k^H sits on l+1.
//
// Layouts (complex, row-major): site i of state b is (D_{i-1}, 2, D_i) at
// sites + b*state_elems + site_off[i]; the row index of (a, s) is 2a + s and
// the column index of (s, c) is s*D + c. Theta is row-major (2 D_{l-1}) x
// (2 D_{l+1}) in theta_buf; its column-major copy in w_buf is the Jacobi
// input.
#include <string.h>

#include "gate_dev.cuh"
#include "gates_dev.cuh"
#include "gemm_tile.cuh"
#include "tnmps_internal.h"

cudaError_t launch_jacobi_gate(tnmps_ctx *c, int l, int Mcap, bool lq);

namespace {

template <typename R>
__device__ __forceinline__ cx<R> *site_ptr(const StateView &v, int b, int i) {
  return reinterpret_cast<cx<R> *>(v.sites) + (int64_t)b * v.state_elems + v.site_off[i];
}
__device__ __forceinline__ int dimv(const StateView &v, int b, int i) {
  return v.dims[(int64_t)b * (v.n + 1) + i];
}

// ---------------------------------------------------------------- init
template <typename R>
__global__ void k_init_state(StateView v, double *discarded) {
  const int b = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= v.n; i += gridDim.x * blockDim.x) {
    v.dims[(int64_t)b * (v.n + 1) + i] = 1;
    if (i < v.n) {
      cx<R> *t = site_ptr<R>(v, b, i);
      t[0] = mkc<R>(1, 0);  // |0>
      t[1] = mkc<R>(0, 0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) discarded[b] = 0.0;
}

// ---------------------------------------------------------------- K2
// X = C_l (2Dl x Dm) * B_{l+1} (Dm x 2Dr) -> theta_buf (row-major, ld 2Dr)
template <typename R>
struct ProbTheta {
  StateView v;
  int l;
  cx<R> *out;
  int64_t tw;
  const cx<R> *A, *B;
  cx<R> *C;
  int lda, ldb, ldc;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M, int &N, int &K) {
    const int Dl = dimv(v, z, l), Dm = dimv(v, z, l + 1), Dr = dimv(v, z, l + 2);
    M = 2 * Dl;
    N = 2 * Dr;
    K = Dm;
    A = site_ptr<R>(v, z, l);
    B = site_ptr<R>(v, z, l + 1);
    C = out + (int64_t)z * tw;
    lda = Dm;
    ldb = 2 * Dr;
    ldc = N;
    return true;
  }
  __device__ cx<R> a(int i, int k) const { return A[(int64_t)i * lda + k]; }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * ldb + j]; }
  __device__ void store(int i, int j, cx<R> val) const { C[(int64_t)i * ldc + j] = val; }
};

// Theta = G X on the physical pair; writes theta_buf (in place) and, unless
// wbuf is null, the column-major Jacobi copy in w_buf. A CTA takes a in
// [a0, a0+16) and every column tile c in [c0, c0+32), i.e. Theta rows
// 2a0..2a0+31 and columns c0.. and Dr+c0.. of both physical halves (the gate,
// built in FP64 from the state's angles, once per CTA): the row-major result
// goes back along rows, and W is written column by column from a
// shared-memory transpose of the tile.
template <typename R>
__global__ void __launch_bounds__(256) k_apply_gate4(StateView v, Op2 op, const double *theta,
                                                           int64_t ths, cx<R> *tbuf, cx<R> *wbuf,
                                                           int64_t tw) {
  const int b = blockIdx.z;
  __shared__ cx<R> G[16];
  __shared__ cx<R> Ts[64][33];  // [column s2*32 + cc][row 2*aa + s1]
  const int l = op.l;
  const int Dl = dimv(v, b, l), Dr = dimv(v, b, l + 2);
  const int a0 = blockIdx.y * 16;
  if (a0 >= Dl) return;  // uniform over the CTA
  if (threadIdx.x == 0) {
    cx<double> Gd[16];
    op2_matrix(op, theta ? theta + (int64_t)b * ths : nullptr, Gd);
    for (int e = 0; e < 16; ++e) G[e] = mkc<R>((R)Gd[e].re, (R)Gd[e].im);
  }
  __syncthreads();
  const int M = 2 * Dl, N = 2 * Dr;
  cx<R> *T = tbuf + (int64_t)b * tw;
  const bool copy = wbuf != nullptr;  // no copy when the Jacobi input is L of Theta = L Q^H
  for (int c0 = 0; c0 < Dr; c0 += 32) {
    for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
      const int aa = e >> 5, cc = e & 31;
      const int a = a0 + aa, c = c0 + cc;
      if (a >= Dl || c >= Dr) continue;
      cx<R> x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = T[(int64_t)(2 * a + (q >> 1)) * N + (q & 1) * Dr + c];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        cx<R> acc = mkc<R>(0, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) cfma(acc, G[4 * r + q], x[q]);
        T[(int64_t)(2 * a + (r >> 1)) * N + (r & 1) * Dr + c] = acc;
        if (copy) Ts[(r & 1) * 32 + cc][2 * aa + (r >> 1)] = acc;
      }
    }
    if (!copy) continue;  // uniform over the CTA
    __syncthreads();
    cx<R> *W = wbuf + (int64_t)b * tw;
    const int rows = min(32, M - 2 * a0), cols = min(32, Dr - c0);
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
      const int jl = e >> 5, il = e & 31;
      const int s2 = jl >> 5, cc = jl & 31;
      if (il < rows && cc < cols)
        W[(int64_t)(s2 * Dr + c0 + cc) * M + 2 * a0 + il] = Ts[jl][il];
    }
    __syncthreads();  // Ts is refilled by the next column tile
  }
}

// ---------------------------------------------------------------- K4
template <typename R>
__global__ void __launch_bounds__(256) k_split_select(StateView v, int l, const cx<R> *wbuf,
                                                      int64_t tw, double eps, double floor_eps,
                                                      int cap, double *discarded, double *scale,
                                                      uint32_t *err,
                                                      unsigned long long *counters) {
  const int b = blockIdx.x;
  const int Dl = dimv(v, b, l), Dm = dimv(v, b, l + 1), Dr = dimv(v, b, l + 2);
  // the Jacobi noise floor (8u of the norm) is always cut: columns below it
  // were not orthogonalised
  const double e_eff = eps > floor_eps ? eps : floor_eps;
  double w;
  bool bad;
  const int k = gdev::select_cta<R>(wbuf + (int64_t)b * tw, 2 * Dl, 2 * Dr, cap, e_eff,
                                    site_ptr<R>(v, b, l), &w, &bad);
  if (threadIdx.x == 0) {
    if (bad) atomicOr(err, TNMPS_EFLAG_NUMERIC);
    discarded[b] += w;
    scale[b] = 1.0;
    v.dims[(int64_t)b * (v.n + 1) + l + 1] = k;
    atomicAdd(&counters[CNT_GATES2Q], 1ull);
    if (Dl == v.chi && Dm == v.chi && Dr == v.chi) atomicAdd(&counters[CNT_GATES2Q_FULL], 1ull);
  }
}

// C_{l+1} (k x 2Dr) = A_l^H (k x M) Theta (M x 2Dr); normalised afterwards
template <typename R>
struct ProbSplit {
  StateView v;
  int l;
  const cx<R> *tb;
  int64_t tw;
  const cx<R> *A, *T;
  cx<R> *C;
  int k, N;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Dl = dimv(v, z, l), Dr = dimv(v, z, l + 2);
    k = dimv(v, z, l + 1);
    N = 2 * Dr;
    M_ = k;
    N_ = N;
    K_ = 2 * Dl;
    A = site_ptr<R>(v, z, l);
    T = tb + (int64_t)z * tw;
    C = site_ptr<R>(v, z, l + 1);
    return true;
  }
  __device__ cx<R> a(int r, int i) const { return cconj(A[(int64_t)i * k + r]); }
  __device__ cx<R> b(int i, int j) const { return T[(int64_t)i * N + j]; }
  __device__ void store(int r, int j, cx<R> val) const { C[(int64_t)r * N + j] = val; }
};

// complex64 form: E = U^H U - I, the FP64 Gram of the orthogonalisation step:
// FP32 FMAs within each 16-wide slice of K, slice sums added in FP64 (see
// gemm_tile_mixed), which keeps the error near 1e-8 for unit columns
struct ProbGram {
  StateView v;
  int l;
  cx<double> *ebuf;
  int64_t estride;
  const cx<float> *U;
  cx<double> *E;
  int k;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    if (blockIdx.y > blockIdx.x) return false;  // Hermitian: upper tiles only, mirrored
    k = dimv(v, z, l + 1);
    M_ = k;
    N_ = k;
    K_ = 2 * dimv(v, z, l);
    U = site_ptr<float>(v, z, l);
    E = ebuf + (int64_t)z * estride;
    return true;
  }
  __device__ cx<float> a(int q, int i) const { return cconj(U[(int64_t)i * k + q]); }
  __device__ cx<float> b(int i, int q) const { return U[(int64_t)i * k + q]; }
  // one writer per entry pair: the upper triangle stores both mirror
  // entries (a diagonal tile also computes the lower ones, rounded
  // differently); the diagonal of a Hermitian Gram is real
  __device__ void store(int q, int r, cx<double> val) const {
    if (q > r) return;
    if (q == r) {
      E[(int64_t)q * k + q] = mkc<double>(val.re - 1.0, 0.0);
      return;
    }
    E[(int64_t)q * k + r] = val;
    E[(int64_t)r * k + q] = cconj(val);
  }
};

// U' = U (I - E/2) -> w_buf (M x k row-major): first-order re-orthonormalisation
struct ProbOrtho {
  StateView v;
  int l;
  const cx<double> *ebuf;
  int64_t estride;
  cx<float> *wbuf;
  int64_t tw;
  const cx<float> *U;
  const cx<double> *E;
  cx<float> *O;
  int k;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    k = dimv(v, z, l + 1);
    M_ = 2 * dimv(v, z, l);
    N_ = k;
    K_ = k;
    U = site_ptr<float>(v, z, l);
    E = ebuf + (int64_t)z * estride;
    O = wbuf + (int64_t)z * tw;
    return true;
  }
  __device__ cx<float> a(int i, int q) const { return U[(int64_t)i * k + q]; }
  __device__ cx<float> b(int q, int r) const {
    const cx<double> e = E[(int64_t)q * k + r];
    return mkc<float>((float)((q == r ? 1.0 : 0.0) - 0.5 * e.re), (float)(-0.5 * e.im));
  }
  __device__ void store(int i, int r, cx<float> val) const { O[(int64_t)i * k + r] = val; }
};

// A_l <- w_buf (M x k)
__global__ void k_copy_u(StateView v, int l, const cx<float> *wbuf, int64_t tw) {
  const int b = blockIdx.y;
  const int cnt = 2 * dimv(v, b, l) * dimv(v, b, l + 1);
  cx<float> *A = site_ptr<float>(v, b, l);
  const cx<float> *W = wbuf + (int64_t)b * tw;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x)
    A[e] = W[e];
}

// scale site tensor `site` of every state to unit Frobenius norm (FP64 sum):
// the new orthogonality centre carries the whole (renormalised) state
template <typename R>
__global__ void __launch_bounds__(256) k_normalise_site(StateView v, int site) {
  const int b = blockIdx.x;
  gdev::normalise_cta<R>(site_ptr<R>(v, b, site), dimv(v, b, site) * 2 * dimv(v, b, site + 1));
}

// ---------------------------------------------------------------- K1
template <typename R>
__global__ void __launch_bounds__(256) k_gate1(StateView v, Op1 op, const double *theta,
                                               int64_t ths) {
  const int b = blockIdx.y;
  __shared__ cx<R> U[4];
  if (threadIdx.x == 0) {
    cx<double> Ud[4];
    side_matrix(op.f, op.nf, theta ? theta + (int64_t)b * ths : nullptr, Ud);
    for (int e = 0; e < 4; ++e) U[e] = mkc<R>((R)Ud[e].re, (R)Ud[e].im);
  }
  __syncthreads();
  const int Dl = dimv(v, b, op.site), Dr = dimv(v, b, op.site + 1);
  cx<R> *X = site_ptr<R>(v, b, op.site);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Dl * Dr; e += gridDim.x * blockDim.x) {
    const int a = e / Dr, c = e - a * Dr;
    const cx<R> x0 = X[(int64_t)(2 * a) * Dr + c], x1 = X[(int64_t)(2 * a + 1) * Dr + c];
    cx<R> y0 = mkc<R>(0, 0), y1 = mkc<R>(0, 0);
    cfma(y0, U[0], x0);
    cfma(y0, U[1], x1);
    cfma(y1, U[2], x0);
    cfma(y1, U[3], x1);
    X[(int64_t)(2 * a) * Dr + c] = y0;
    X[(int64_t)(2 * a + 1) * Dr + c] = y1;
  }
}

// ---------------------------------------------------------------- K7
// Householder kernels: two CTAs per SM for complex64 columns of up to 256
// rows; complex128 and longer columns take one, so that the block reflectors'
// columns stay in registers.
// Right move at site c: C_c (2Dl x Dr) = Q R;  A_c <- Q;  R stays in w_buf.
template <typename R, int HR>
__global__ void __launch_bounds__(256, sizeof(R) == 8 || HR > 8 ? 1 : 2)
    k_qr_right(StateView v, int c, cx<R> *wbuf, cx<R> *tbuf, int64_t tw, int32_t *newdim) {
  const int b = blockIdx.x;
  const int r = gdev::qr_right_cta<R, HR>(site_ptr<R>(v, b, c), dimv(v, b, c), dimv(v, b, c + 1),
                                      wbuf + (int64_t)b * tw, tbuf + (int64_t)b * tw);
  if (threadIdx.x == 0) newdim[b] = r;
}

// Left move at site c: C_c (Dl x 2Dr) = L Q via QR of C_c^H = Q' R';
// B_c <- Q'^H,  L = R'^H stays (as R') in w_buf.
template <typename R, int HR>
__global__ void __launch_bounds__(256, sizeof(R) == 8 || HR > 8 ? 1 : 2)
    k_lq_left(StateView v, int c, cx<R> *wbuf, cx<R> *tbuf, int64_t tw, int32_t *newdim) {
  const int b = blockIdx.x;
  const int r = gdev::lq_left_cta<R, HR>(site_ptr<R>(v, b, c), dimv(v, b, c), dimv(v, b, c + 1),
                                     wbuf + (int64_t)b * tw, tbuf + (int64_t)b * tw);
  if (threadIdx.x == 0) newdim[b] = r;
}

// K3 preconditioner: Theta (theta_buf, row-major 2D_{l-1} x 2D_{l+1}) = L Q^H;
// L (column-major, the Jacobi input) -> w_buf, Householder scratch in qbuf.
template <typename R, int HR>
__global__ void __launch_bounds__(256, sizeof(R) == 8 || HR > 8 ? 1 : 2)
    k_lq_theta(StateView v, int l, const cx<R> *tbuf, cx<R> *qbuf, cx<R> *wbuf, int64_t tw) {
  const int b = blockIdx.x;
  gdev::lq_theta_cta<R, HR>(tbuf + (int64_t)b * tw, 2 * dimv(v, b, l), 2 * dimv(v, b, l + 2),
                            qbuf + (int64_t)b * tw, wbuf + (int64_t)b * tw);
}

// out (r x 2D') = R (r x Dr, upper triangle of w_buf, ld 2Dl) * B_{c+1} (Dr x 2D')
template <typename R>
struct ProbRB {
  StateView v;
  int c;
  const cx<R> *wbuf;
  cx<R> *tbuf;
  int64_t tw;
  const int32_t *newdim;
  const cx<R> *Wm, *B;
  cx<R> *O;
  int m, N;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Dl = dimv(v, z, c), Dr = dimv(v, z, c + 1), D2 = dimv(v, z, c + 2);
    m = 2 * Dl;
    N = 2 * D2;
    M_ = newdim[z];
    N_ = N;
    K_ = Dr;
    Wm = wbuf + (int64_t)z * tw;
    B = site_ptr<R>(v, z, c + 1);
    O = tbuf + (int64_t)z * tw;
    return true;
  }
  __device__ cx<R> a(int q, int k) const {
    return k >= q ? Wm[(int64_t)k * m + q] : mkc<R>(0, 0);
  }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * N + j]; }
  __device__ void store(int q, int j, cx<R> val) const { O[(int64_t)q * N + j] = val; }
};

// out (2D'' x r) = A_{c-1} (2D'' x Dl) * L (Dl x r), L[k][q] = conj(R'[q][k])
template <typename R>
struct ProbAL {
  StateView v;
  int c;
  const cx<R> *wbuf;
  cx<R> *tbuf;
  int64_t tw;
  const int32_t *newdim;
  const cx<R> *Wm, *A;
  cx<R> *O;
  int m, Dl, r;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int D0 = dimv(v, z, c - 1);
    Dl = dimv(v, z, c);
    m = 2 * dimv(v, z, c + 1);
    r = newdim[z];
    M_ = 2 * D0;
    N_ = r;
    K_ = Dl;
    Wm = wbuf + (int64_t)z * tw;
    A = site_ptr<R>(v, z, c - 1);
    O = tbuf + (int64_t)z * tw;
    return true;
  }
  __device__ cx<R> a(int i, int k) const { return A[(int64_t)i * Dl + k]; }
  __device__ cx<R> b(int k, int q) const {
    return k >= q ? cconj(Wm[(int64_t)k * m + q]) : mkc<R>(0, 0);
  }
  __device__ void store(int i, int q, cx<R> val) const { O[(int64_t)i * r + q] = val; }
};

// site `dst` <- tbuf (elements = rows * cols), then dims[b][bond] = newdim[b]
template <typename R>
__global__ void k_copy_site(StateView v, int dst, int bond, int rows_idx, int cols_idx,
                            bool rows_from_new, const cx<R> *tbuf, int64_t tw,
                            const int32_t *newdim) {
  const int b = blockIdx.y;
  const int nd = newdim[b];
  const int rows = rows_from_new ? nd : 2 * dimv(v, b, rows_idx);
  const int cols = rows_from_new ? 2 * dimv(v, b, cols_idx) : nd;
  const int64_t cnt = (int64_t)rows * cols;
  cx<R> *X = site_ptr<R>(v, b, dst);
  const cx<R> *T = tbuf + (int64_t)b * tw;
  for (int64_t e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x)
    X[e] = T[e];
}

__global__ void k_set_bond(StateView v, int bond, const int32_t *newdim) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < v.batch) v.dims[(int64_t)b * (v.n + 1) + bond] = newdim[b];
}

template <typename R>
cudaError_t split_impl(tnmps_ctx *c, const Op2 &op, const double *theta, int64_t ths,
                       cudaEvent_t ev);

template <typename R>
cudaError_t gate2_impl(tnmps_ctx *c, const Op2 &op, const double *theta, int64_t ths) {
  const StateView v = c->view();
  const int l = op.l;
  const int Mmax = 2 * c->ub[l], Nmax = 2 * c->ub[l + 2];
  cx<R> *tb = reinterpret_cast<cx<R> *>(c->theta_buf);
  cx<R> *wb = reinterpret_cast<cx<R> *>(c->w_buf);
  cudaError_t e;
  // K2: Theta = G (C_l B_{l+1})
  cudaEvent_t ev = prof_begin(c, PC_THETA);
  if (c->dtype == TNMPS_C64_BF16SPLIT) {  // tensor cores, BF16 split products
    if ((e = launch_theta_tc(c, l)) != cudaSuccess) return e;
  } else {
    ProbTheta<R> pt{};
    pt.v = v;
    pt.l = l;
    pt.out = tb;
    pt.tw = c->tw;
    if ((e = launch_gemm<R>(pt, Mmax, Nmax, c->batch, c->stream, &c->launches)) != cudaSuccess)
      return e;
  }
  return split_impl<R>(c, op, theta, ths, ev);
}

// G applied to the block in theta_buf (row-major, 2D_{l-1} x 2D_{l+1}), then
// K3 (Jacobi) and K4 (rank by rule R under the bond cap, A_l <- U_k,
// C_{l+1} <- U_k^H Theta, normalised); the centre ends on l+1. ev: open
// PC_THETA timing event of the caller (or null).
template <typename R>
cudaError_t split_impl(tnmps_ctx *c, const Op2 &op, const double *theta, int64_t ths,
                       cudaEvent_t ev) {
  const StateView v = c->view();
  const int l = op.l;
  const int Mmax = 2 * c->ub[l], Nmax = 2 * c->ub[l + 2];
  cx<R> *tb = reinterpret_cast<cx<R> *>(c->theta_buf);
  cx<R> *wb = reinterpret_cast<cx<R> *>(c->w_buf);
  cudaError_t e;
  {
    dim3 grid(1, (c->ub[l] + 15) / 16, c->batch);  // a CTA loops over the column tiles
    k_apply_gate4<R><<<grid, 256, 0, c->stream>>>(v, op, theta, ths, tb, c->svd_lq ? nullptr : wb,
                                                   c->tw);
    ++c->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_end(c, PC_THETA, ev);
  if (c->svd_lq) {  // Theta = L Q^H: the Jacobi input becomes L (same sigma and U)
    ev = prof_begin(c, PC_SVD_LQ);
    cx<R> *qb = reinterpret_cast<cx<R> *>(c->q_buf);
    if (Nmax <= 256)
      k_lq_theta<R, 8><<<c->batch, 256, 0, c->stream>>>(v, l, tb, qb, wb, c->tw);
    else
      k_lq_theta<R, 16><<<c->batch, 256, 0, c->stream>>>(v, l, tb, qb, wb, c->tw);
    ++c->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_end(c, PC_SVD_LQ, ev);
  }
  // K3: one-sided Jacobi on the column-major copy (or on L)
  ev = prof_begin(c, PC_JACOBI);
  if ((e = launch_jacobi_gate(c, l, Mmax, c->svd_lq != 0)) != cudaSuccess) return e;
  ++c->launches;
  prof_end(c, PC_JACOBI, ev);
  // K4: rank, A_l <- U_k, [orthonormalise U_k], C_{l+1} <- U_k^H Theta, normalise
  ev = prof_begin(c, PC_SPLIT);
  const double floor_eps =
      c->dtype != TNMPS_C128 ? 8.0 * 5.9604644775390625e-08 : 8.0 * 1.1102230246251565e-16;
  int cap = c->cap[l + 1];
  if (c->fit_cap > 0 && c->fit_cap < cap) cap = c->fit_cap;
  k_split_select<R><<<c->batch, 256, 0, c->stream>>>(v, l, wb, c->tw, c->eps, floor_eps, cap,
                                                      c->discarded, c->scale, c->err,
                                                      c->counters);
  ++c->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int kub = cap;
  kub = kub < Mmax ? kub : Mmax;
  kub = kub < Nmax ? kub : Nmax;
  if (sizeof(R) == 4) {
    ProbGram pg{};
    pg.v = v;
    pg.l = l;
    pg.ebuf = reinterpret_cast<cx<double> *>(c->ebuf);
    pg.estride = (int64_t)c->chi * c->chi;
    if ((e = launch_gemm_mixed(pg, kub, kub, c->batch, c->stream, &c->launches)) != cudaSuccess)
      return e;
    ProbOrtho po{};
    po.v = v;
    po.l = l;
    po.ebuf = pg.ebuf;
    po.estride = pg.estride;
    po.wbuf = reinterpret_cast<cx<float> *>(c->w_buf);
    po.tw = c->tw;
    if ((e = launch_gemm<float>(po, Mmax, kub, c->batch, c->stream, &c->launches)) != cudaSuccess)
      return e;
    dim3 grid((Mmax * kub + 255) / 256, c->batch);
    k_copy_u<<<grid, 256, 0, c->stream>>>(v, l, reinterpret_cast<cx<float> *>(c->w_buf), c->tw);
    ++c->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (c->dtype == TNMPS_C64_BF16SPLIT) {  // tensor cores, three BF16 pieces
    if ((e = launch_split_tc(c, l, kub)) != cudaSuccess) return e;
  } else {
    ProbSplit<R> ps{};
    ps.v = v;
    ps.l = l;
    ps.tb = tb;
    ps.tw = c->tw;
    if ((e = launch_gemm<R>(ps, kub, Nmax, c->batch, c->stream, &c->launches)) != cudaSuccess)
      return e;
  }
  k_normalise_site<R><<<c->batch, 256, 0, c->stream>>>(v, l + 1);
  ++c->launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_end(c, PC_SPLIT, ev);
  c->ub[l + 1] = kub;
  return cudaSuccess;
}

template <typename R>
cudaError_t move_right_impl(tnmps_ctx *c, int s) {
  const StateView v = c->view();
  cx<R> *tb = reinterpret_cast<cx<R> *>(c->theta_buf);
  cx<R> *wb = reinterpret_cast<cx<R> *>(c->w_buf);
  cudaEvent_t ev = prof_begin(c, PC_MOVE);
  // block reflectors hold a column's rows in registers: 8 per lane up to 256 rows
  if (2 * c->chi <= 256)
    k_qr_right<R, 8><<<c->batch, 256, 0, c->stream>>>(v, s, wb, tb, c->tw, c->perm);
  else
    k_qr_right<R, 16><<<c->batch, 256, 0, c->stream>>>(v, s, wb, tb, c->tw, c->perm);
  c->launches += 4;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int rub = 2 * c->ub[s];
  rub = rub < c->ub[s + 1] ? rub : c->ub[s + 1];
  ProbRB<R> p{};
  p.v = v;
  p.c = s;
  p.wbuf = wb;
  p.tbuf = tb;
  p.tw = c->tw;
  p.newdim = c->perm;
  if ((e = launch_gemm<R>(p, rub, 2 * c->ub[s + 2], c->batch, c->stream)) != cudaSuccess) return e;
  const int64_t cnt = (int64_t)rub * 2 * c->ub[s + 2];
  dim3 grid((unsigned)((cnt + 255) / 256), c->batch);
  k_copy_site<R><<<grid, 256, 0, c->stream>>>(v, s + 1, s + 1, 0, s + 2, true, tb, c->tw, c->perm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_set_bond<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(v, s + 1, c->perm);
  prof_end(c, PC_MOVE, ev);
  c->ub[s + 1] = rub;
  return cudaGetLastError();
}

template <typename R>
cudaError_t move_left_impl(tnmps_ctx *c, int s) {
  const StateView v = c->view();
  cx<R> *tb = reinterpret_cast<cx<R> *>(c->theta_buf);
  cx<R> *wb = reinterpret_cast<cx<R> *>(c->w_buf);
  cudaEvent_t ev = prof_begin(c, PC_MOVE);
  if (2 * c->chi <= 256)
    k_lq_left<R, 8><<<c->batch, 256, 0, c->stream>>>(v, s, wb, tb, c->tw, c->perm);
  else
    k_lq_left<R, 16><<<c->batch, 256, 0, c->stream>>>(v, s, wb, tb, c->tw, c->perm);
  c->launches += 4;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int rub = 2 * c->ub[s + 1];
  rub = rub < c->ub[s] ? rub : c->ub[s];
  ProbAL<R> p{};
  p.v = v;
  p.c = s;
  p.wbuf = wb;
  p.tbuf = tb;
  p.tw = c->tw;
  p.newdim = c->perm;
  if ((e = launch_gemm<R>(p, 2 * c->ub[s - 1], rub, c->batch, c->stream)) != cudaSuccess) return e;
  const int64_t cnt = (int64_t)2 * c->ub[s - 1] * rub;
  dim3 grid((unsigned)((cnt + 255) / 256), c->batch);
  k_copy_site<R><<<grid, 256, 0, c->stream>>>(v, s - 1, s, s - 1, 0, false, tb, c->tw, c->perm);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_set_bond<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(v, s, c->perm);
  prof_end(c, PC_MOVE, ev);
  c->ub[s] = rub;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_state(tnmps_ctx *c) {
  dim3 grid((c->n + 1 + 255) / 256, c->batch);
  ++c->launches;
  if (c->dtype == TNMPS_C128)
    k_init_state<double><<<grid, 256, 0, c->stream>>>(c->view(), c->discarded);
  else
    k_init_state<float><<<grid, 256, 0, c->stream>>>(c->view(), c->discarded);
  return cudaGetLastError();
}

cudaError_t launch_gate2(tnmps_ctx *c, const Op2 &op, const double *theta, int64_t ths) {
  return c->dtype == TNMPS_C128 ? gate2_impl<double>(c, op, theta, ths)
                                : gate2_impl<float>(c, op, theta, ths);
}

cudaError_t launch_split_theta(tnmps_ctx *c, int l) {
  Op2 op;
  memset(&op, 0, sizeof op);
  op.l = l;
  for (int d = 0; d < 4; ++d) op.core[2 * (4 * d + d)] = 1.0;  // identity 4x4
  return c->dtype == TNMPS_C128 ? split_impl<double>(c, op, nullptr, 0, nullptr)
                                : split_impl<float>(c, op, nullptr, 0, nullptr);
}

cudaError_t launch_gate1(tnmps_ctx *c, const Op1 &op, const double *theta, int64_t ths) {
  const int work = c->ub[op.site] * c->ub[op.site + 1];
  dim3 grid((work + 255) / 256, c->batch);
  ++c->launches;
  if (c->dtype == TNMPS_C128)
    k_gate1<double><<<grid, 256, 0, c->stream>>>(c->view(), op, theta, ths);
  else
    k_gate1<float><<<grid, 256, 0, c->stream>>>(c->view(), op, theta, ths);
  return cudaGetLastError();
}

cudaError_t launch_move_right(tnmps_ctx *c, int s) {
  return c->dtype == TNMPS_C128 ? move_right_impl<double>(c, s) : move_right_impl<float>(c, s);
}

cudaError_t launch_move_left(tnmps_ctx *c, int s) {
  return c->dtype == TNMPS_C128 ? move_left_impl<double>(c, s) : move_left_impl<float>(c, s);
}
