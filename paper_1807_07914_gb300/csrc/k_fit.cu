// Super-gate application by overlap maximisation (Sec. II, the general
// gate-action algorithm; Sec. IV, the ExaTENSOR MPS visitor): the contractions
// of the closed network <TN_out|TN_mid> over the window [p, q] of the
// super-gate, with TN_mid = the input state psi (a snapshot of the window)
// plus the super-gate as an MPO W, and TN_out = phi, the context's state.
//
// Every step is a batched complex GEMM on the shared-memory tile core
// (gemm_tile.cuh); the problem functors below fold the index maps of the
// tensor legs into the operand loads, so no operand is permuted in memory.
//
// Layouts (complex, row-major, per state):
//   phi site i    [D_{i-1}][2][D_i]   (the context's sites)
//   psi site i    same, in the snapshot, at site_off[i] - site_off[p]
//   W site i      [w_{i-1}][2 out][2 in][w_i]  (shared by all states)
//   environment   [D^phi][w][D^psi] on one bond: L_i[b', beta, b] for the
//                 left environments, R_i[c', gamma, c] for the right ones
// Two-site gradient at the pair (i, i+1), with F = phi and P = psi dims:
//   S1 = T1[(a', al), (s1, m)]       = sum_a  L[a', al, a] psi_i[a, s1, m]
//   S2 = T2[(a', s1', be), m]        = sum_{al, s1} W_i[al, s1', s1, be] T1
//   S1 = T3[(a', s1', be), (s2, c)]  = sum_m  T2 psi_{i+1}[m, s2, c]
//   S3 = T4[(a', s1', s2', ga), c]   = sum_{be, s2} W_{i+1}[be, s2', s2, ga] T3
//   Theta[(a', s1'), (s2', c')]      = sum_{ga, c} T4 R[c', ga, c]
// and after the split L_i[b', (be, b)] = sum_{a', s1'} conj(phi_i[a', s1', b']) T2.
// Right environments (R_i from R_{i+1}):
//   S1 = V1[(c, s), (d', de)]        = sum_d  psi_i[c, s, d] R_{i+1}[d', de, d]
//   S2 = V2[(s', d'), (ga, c)]       = sum_{s, de} W_i[ga, s', s, de] V1
//   R_i[c', (ga, c)]                 = sum_{s', d'} conj(phi_i[c', s', d']) V2
#include "gemm_tile.cuh"
#include "tnmps_internal.h"

namespace {

template <typename R>
struct FitBase {
  StateView v;              // phi
  const cx<R> *psi;         // snapshot of psi's window, per state psi_stride elements
  int64_t psi_stride, psi_base;
  const int32_t *pdims;     // [batch][n+1] psi dims
  cx<R> *s1, *s2, *s3;      // scratch, per state s_stride elements
  int64_t s_stride;
  cx<R> *env;               // environment slots, per state env_stride elements
  int64_t env_stride;

  __device__ int fd(int z, int i) const { return v.dims[(int64_t)z * (v.n + 1) + i]; }
  __device__ int pd(int z, int i) const { return pdims[(int64_t)z * (v.n + 1) + i]; }
  __device__ cx<R> *phi_site(int z, int i) const {
    return reinterpret_cast<cx<R> *>(v.sites) + (int64_t)z * v.state_elems + v.site_off[i];
  }
  __device__ const cx<R> *psi_site(int z, int i) const {
    return psi + (int64_t)z * psi_stride + (v.site_off[i] - psi_base);
  }
  __device__ cx<R> *S1(int z) const { return s1 + (int64_t)z * s_stride; }
  __device__ cx<R> *S2(int z) const { return s2 + (int64_t)z * s_stride; }
  __device__ cx<R> *S3(int z) const { return s3 + (int64_t)z * s_stride; }
  __device__ cx<R> *E(int z, int64_t off) const { return env + (int64_t)z * env_stride + off; }
};

// T1 = L (Fa wa x Pa) psi_i (Pa x 2Pm)
template <typename R>
struct FitT1 : FitBase<R> {
  int i, wa;
  int64_t el;
  const cx<R> *A, *B;
  cx<R> *C;
  int K, N;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i), Pa = this->pd(z, i), Pm = this->pd(z, i + 1);
    M_ = Fa * wa;
    N_ = N = 2 * Pm;
    K_ = K = Pa;
    A = this->E(z, el);
    B = this->psi_site(z, i);
    C = this->S1(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return A[(int64_t)r * K + k]; }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * N + j]; }
  __device__ void store(int r, int j, cx<R> x) const { C[(int64_t)r * N + j] = x; }
};

// T2[(a', s', be), m] = sum_{al, s} W[al, s', s, be] T1[(a', al), (s, m)]
// as a GEMM: rows (s', be), columns (a', m), k = (al, s)
template <typename R>
struct FitT2 : FitBase<R> {
  int i, wa, wm;
  const cx<R> *W;
  const cx<R> *B;
  cx<R> *C;
  int Pm;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i);
    Pm = this->pd(z, i + 1);
    M_ = 2 * wm;
    N_ = Fa * Pm;
    K_ = 2 * wa;
    B = this->S1(z);
    C = this->S2(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const {
    const int sp = r / wm, be = r - sp * wm, al = k >> 1, s = k & 1;
    return W[((al * 2 + sp) * 2 + s) * wm + be];
  }
  __device__ cx<R> b(int k, int j) const {
    const int al = k >> 1, s = k & 1, ap = j / Pm, m = j - ap * Pm;
    return B[((int64_t)ap * wa + al) * 2 * Pm + s * Pm + m];
  }
  __device__ void store(int r, int j, cx<R> x) const {
    const int sp = r / wm, be = r - sp * wm, ap = j / Pm, m = j - ap * Pm;
    C[(((int64_t)ap * 2 + sp) * wm + be) * Pm + m] = x;
  }
};

// T3 = T2 (Fa 2 wm x Pm) psi_{i+1} (Pm x 2Pc)
template <typename R>
struct FitT3 : FitBase<R> {
  int i, wm;
  const cx<R> *A, *B;
  cx<R> *C;
  int K, N;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i), Pm = this->pd(z, i + 1), Pc = this->pd(z, i + 2);
    M_ = Fa * 2 * wm;
    N_ = N = 2 * Pc;
    K_ = K = Pm;
    A = this->S2(z);
    B = this->psi_site(z, i + 1);
    C = this->S1(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return A[(int64_t)r * K + k]; }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * N + j]; }
  __device__ void store(int r, int j, cx<R> x) const { C[(int64_t)r * N + j] = x; }
};

// T4[(a', s1', s2', ga), c] = sum_{be, s2} W2[be, s2', s2, ga] T3[(a', s1', be), (s2, c)]
// as a GEMM: rows (s2', ga), columns (a' s1', c), k = (be, s2)
template <typename R>
struct FitT4 : FitBase<R> {
  int i, wm, wc;
  const cx<R> *W;
  const cx<R> *B;
  cx<R> *C;
  int Pc;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i);
    Pc = this->pd(z, i + 2);
    M_ = 2 * wc;
    N_ = 2 * Fa * Pc;
    K_ = 2 * wm;
    B = this->S1(z);
    C = this->S3(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const {
    const int sp = r / wc, ga = r - sp * wc, be = k >> 1, s = k & 1;
    return W[((be * 2 + sp) * 2 + s) * wc + ga];
  }
  __device__ cx<R> b(int k, int j) const {
    const int be = k >> 1, s = k & 1, as = j / Pc, c = j - as * Pc;
    return B[((int64_t)as * wm + be) * 2 * Pc + s * Pc + c];
  }
  __device__ void store(int r, int j, cx<R> x) const {
    const int sp = r / wc, ga = r - sp * wc, as = j / Pc, c = j - as * Pc;
    C[(((int64_t)as * 2 + sp) * wc + ga) * Pc + c] = x;
  }
};

// Theta[(a' s1'), (s2' c')] = sum_{(ga, c)} T4[(a' s1' s2'), (ga, c)] R[c', (ga, c)]
// rows r = (a' s1' s2') of T4, stored at theta row r >> 1, column (r & 1) Fc + c'
template <typename R>
struct FitTheta : FitBase<R> {
  int i, wc;
  int64_t er;
  cx<R> *tb;
  int64_t tw;
  const cx<R> *A, *B;
  cx<R> *C;
  int K, Fc;
  static constexpr bool A_KFAST = true, B_KFAST = true;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i), Pc = this->pd(z, i + 2);
    Fc = this->fd(z, i + 2);
    M_ = 4 * Fa;
    N_ = Fc;
    K_ = K = wc * Pc;
    A = this->S3(z);
    B = this->E(z, er);
    C = tb + (int64_t)z * tw;
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return A[(int64_t)r * K + k]; }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)j * K + k]; }
  __device__ void store(int r, int j, cx<R> x) const {
    C[(int64_t)(r >> 1) * 2 * Fc + (r & 1) * Fc + j] = x;
  }
};

// L_i[b', (be, b)] = sum_{(a' s')} conj(phi_i[(a' s'), b']) T2[(a' s'), (be, b)]
template <typename R>
struct FitEnvL : FitBase<R> {
  int i, wm;
  int64_t eo;
  const cx<R> *A, *B;
  cx<R> *C;
  int Fm, N;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i), Pm = this->pd(z, i + 1);
    Fm = this->fd(z, i + 1);
    M_ = Fm;
    N_ = N = wm * Pm;
    K_ = 2 * Fa;
    A = this->phi_site(z, i);
    B = this->S2(z);
    C = this->E(z, eo);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return cconj(A[(int64_t)k * Fm + r]); }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * N + j]; }
  __device__ void store(int r, int j, cx<R> x) const { C[(int64_t)r * N + j] = x; }
};

// V1[(c, s), (d', de)] = sum_d psi_i[(c, s), d] R_{i+1}[(d', de), d]
template <typename R>
struct FitV1 : FitBase<R> {
  int i, wm;
  int64_t er;
  const cx<R> *A, *B;
  cx<R> *C;
  int K, N;
  static constexpr bool A_KFAST = true, B_KFAST = true;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Pa = this->pd(z, i), Pm = this->pd(z, i + 1), Fm = this->fd(z, i + 1);
    M_ = 2 * Pa;
    N_ = N = Fm * wm;
    K_ = K = Pm;
    A = this->psi_site(z, i);
    B = this->E(z, er);
    C = this->S1(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return A[(int64_t)r * K + k]; }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)j * K + k]; }
  __device__ void store(int r, int j, cx<R> x) const { C[(int64_t)r * N + j] = x; }
};

// V2[(s', d'), (ga, c)] = sum_{(s, de)} W[(ga, s'), (s, de)] V1[(c, s), (d', de)]
// as a GEMM: rows (ga, s'), columns (c, d'), k = (s, de)
template <typename R>
struct FitV2 : FitBase<R> {
  int i, wa, wm;
  const cx<R> *W;
  const cx<R> *B;
  cx<R> *C;
  int Fm, Pa;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    Pa = this->pd(z, i);
    Fm = this->fd(z, i + 1);
    M_ = 2 * wa;
    N_ = Pa * Fm;
    K_ = 2 * wm;
    B = this->S1(z);
    C = this->S2(z);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return W[r * 2 * wm + k]; }
  __device__ cx<R> b(int k, int j) const {
    const int s = k / wm, de = k - s * wm, c = j / Fm, dp = j - c * Fm;
    return B[((int64_t)c * 2 + s) * Fm * wm + (int64_t)dp * wm + de];
  }
  __device__ void store(int r, int j, cx<R> x) const {
    const int ga = r >> 1, sp = r & 1, c = j / Fm, dp = j - c * Fm;
    C[((int64_t)sp * Fm + dp) * wa * Pa + (int64_t)ga * Pa + c] = x;
  }
};

// R_i[c', (ga, c)] = sum_{(s', d')} conj(phi_i[c', (s', d')]) V2[(s', d'), (ga, c)]
template <typename R>
struct FitEnvR : FitBase<R> {
  int i, wa;
  int64_t eo;
  const cx<R> *A, *B;
  cx<R> *C;
  int K, N;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M_, int &N_, int &K_) {
    const int Fa = this->fd(z, i), Fm = this->fd(z, i + 1), Pa = this->pd(z, i);
    M_ = Fa;
    N_ = N = wa * Pa;
    K_ = K = 2 * Fm;
    A = this->phi_site(z, i);
    B = this->S2(z);
    C = this->E(z, eo);
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return cconj(A[(int64_t)r * K + k]); }
  __device__ cx<R> b(int k, int j) const { return B[(int64_t)k * N + j]; }
  __device__ void store(int r, int j, cx<R> x) const { C[(int64_t)r * N + j] = x; }
};

// identity environment on a window boundary bond (w = 1, D^phi = D^psi = D)
template <typename R>
__global__ void k_env_identity(FitBase<R> fb, int dims_index, int64_t off) {
  const int z = blockIdx.y;
  const int D = fb.fd(z, dims_index);
  cx<R> *E = fb.E(z, off);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < D * D; e += gridDim.x * blockDim.x) {
    const int r = e / D, c = e - r * D;
    E[(int64_t)r * D + c] = mkc<R>(r == c ? 1 : 0, 0);
  }
}

// O_z = sum_b L_q[b, 0, b] (w = 1 and D^phi = D^psi on the bond right of the window)
template <typename R>
__global__ void k_env_trace(FitBase<R> fb, int dims_index, int64_t off, double *out) {
  const int z = blockIdx.x;
  const int D = fb.fd(z, dims_index);
  const cx<R> *E = fb.E(z, off);
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < D; b += blockDim.x) {
    const cx<R> x = E[(int64_t)b * D + b];
    re += (double)x.re;
    im += (double)x.im;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sr[threadIdx.x] += sr[threadIdx.x + o];
      si[threadIdx.x] += si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * z] = sr[0];
    out[2 * z + 1] = si[0];
  }
}

// discarded_z = saved_z + max(0, 1 - |O_z|^2)
__global__ void k_fit_finish(const double *saved, const double *ov, double *discarded, int batch) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= batch) return;
  const double f = ov[2 * z] * ov[2 * z] + ov[2 * z + 1] * ov[2 * z + 1];
  discarded[z] = saved[z] + (f < 1.0 ? 1.0 - f : 0.0);
}

template <typename R>
FitBase<R> base_of(tnmps_ctx *c, const FitDev &f) {
  FitBase<R> b;
  b.v = c->view();
  b.psi = reinterpret_cast<const cx<R> *>(f.psi);
  b.psi_stride = f.psi_stride;
  b.psi_base = f.psi_base;
  b.pdims = f.pdims;
  b.s1 = reinterpret_cast<cx<R> *>(f.s1);
  b.s2 = reinterpret_cast<cx<R> *>(f.s2);
  b.s3 = reinterpret_cast<cx<R> *>(f.s3);
  b.s_stride = f.s_stride;
  b.env = reinterpret_cast<cx<R> *>(f.env);
  b.env_stride = f.env_stride;
  return b;
}

template <typename R>
const cx<R> *mpo_site(const FitDev &f, int i) {
  return reinterpret_cast<const cx<R> *>(f.mpo) + f.mpo_off[i - f.p];
}

template <typename R>
cudaError_t pair_grad(tnmps_ctx *c, const FitDev &f, int i) {
  const FitBase<R> fb = base_of<R>(c, f);
  const int wa = f.w[i - f.p], wm = f.w[i - f.p + 1], wc = f.w[i - f.p + 2];
  const int Fa = c->ub[i], Fc = c->ub[i + 2];
  const int Pa = f.pub[i], Pm = f.pub[i + 1], Pc = f.pub[i + 2];
  uint64_t *L = &c->launches;
  cudaError_t e;
  FitT1<R> t1{};
  static_cast<FitBase<R> &>(t1) = fb;
  t1.i = i;
  t1.wa = wa;
  t1.el = f.env_off[i - f.p];  // bond i-1
  if ((e = launch_gemm<R>(t1, Fa * wa, 2 * Pm, c->batch, c->stream, L)) != cudaSuccess) return e;
  FitT2<R> t2{};
  static_cast<FitBase<R> &>(t2) = fb;
  t2.i = i;
  t2.wa = wa;
  t2.wm = wm;
  t2.W = mpo_site<R>(f, i);
  if ((e = launch_gemm<R>(t2, 2 * wm, Fa * Pm, c->batch, c->stream, L)) != cudaSuccess) return e;
  FitT3<R> t3{};
  static_cast<FitBase<R> &>(t3) = fb;
  t3.i = i;
  t3.wm = wm;
  if ((e = launch_gemm<R>(t3, Fa * 2 * wm, 2 * Pc, c->batch, c->stream, L)) != cudaSuccess)
    return e;
  FitT4<R> t4{};
  static_cast<FitBase<R> &>(t4) = fb;
  t4.i = i;
  t4.wm = wm;
  t4.wc = wc;
  t4.W = mpo_site<R>(f, i + 1);
  if ((e = launch_gemm<R>(t4, 2 * wc, 2 * Fa * Pc, c->batch, c->stream, L)) != cudaSuccess)
    return e;
  FitTheta<R> th{};
  static_cast<FitBase<R> &>(th) = fb;
  th.i = i;
  th.wc = wc;
  th.er = f.env_off[i + 2 - f.p];  // bond i+1
  th.tb = reinterpret_cast<cx<R> *>(c->theta_buf);
  th.tw = c->tw;
  return launch_gemm<R>(th, 4 * Fa, Fc, c->batch, c->stream, L);
}

// T1, T2 at site i, then L_i on bond i from phi_i (which must be final)
template <typename R>
cudaError_t env_left(tnmps_ctx *c, const FitDev &f, int i, bool have_t2) {
  const FitBase<R> fb = base_of<R>(c, f);
  const int wa = f.w[i - f.p], wm = f.w[i - f.p + 1];
  const int Fa = c->ub[i], Fm = c->ub[i + 1];
  const int Pm = f.pub[i + 1];
  uint64_t *L = &c->launches;
  cudaError_t e;
  if (!have_t2) {
    FitT1<R> t1{};
    static_cast<FitBase<R> &>(t1) = fb;
    t1.i = i;
    t1.wa = wa;
    t1.el = f.env_off[i - f.p];
    if ((e = launch_gemm<R>(t1, Fa * wa, 2 * Pm, c->batch, c->stream, L)) != cudaSuccess)
      return e;
    FitT2<R> t2{};
    static_cast<FitBase<R> &>(t2) = fb;
    t2.i = i;
    t2.wa = wa;
    t2.wm = wm;
    t2.W = mpo_site<R>(f, i);
    if ((e = launch_gemm<R>(t2, 2 * wm, Fa * Pm, c->batch, c->stream, L)) != cudaSuccess)
      return e;
  }
  FitEnvL<R> el{};
  static_cast<FitBase<R> &>(el) = fb;
  el.i = i;
  el.wm = wm;
  el.eo = f.env_off[i + 1 - f.p];  // bond i
  return launch_gemm<R>(el, Fm, wm * Pm, c->batch, c->stream, L);
}

// R_i on bond i-1 from R_{i+1} on bond i
template <typename R>
cudaError_t env_right(tnmps_ctx *c, const FitDev &f, int i) {
  const FitBase<R> fb = base_of<R>(c, f);
  const int wa = f.w[i - f.p], wm = f.w[i - f.p + 1];
  const int Fa = c->ub[i], Fm = c->ub[i + 1];
  const int Pa = f.pub[i];
  uint64_t *L = &c->launches;
  cudaError_t e;
  FitV1<R> v1{};
  static_cast<FitBase<R> &>(v1) = fb;
  v1.i = i;
  v1.wm = wm;
  v1.er = f.env_off[i + 1 - f.p];
  if ((e = launch_gemm<R>(v1, 2 * Pa, Fm * wm, c->batch, c->stream, L)) != cudaSuccess) return e;
  FitV2<R> v2{};
  static_cast<FitBase<R> &>(v2) = fb;
  v2.i = i;
  v2.wa = wa;
  v2.wm = wm;
  v2.W = mpo_site<R>(f, i);
  if ((e = launch_gemm<R>(v2, 2 * wa, Pa * Fm, c->batch, c->stream, L)) != cudaSuccess) return e;
  FitEnvR<R> er{};
  static_cast<FitBase<R> &>(er) = fb;
  er.i = i;
  er.wa = wa;
  er.eo = f.env_off[i - f.p];
  return launch_gemm<R>(er, Fa, wa * Pa, c->batch, c->stream, L);
}

template <typename R>
cudaError_t boundary(tnmps_ctx *c, const FitDev &f, int bond) {
  const FitBase<R> fb = base_of<R>(c, f);
  const int D = c->ub[bond + 1];
  dim3 grid((D * D + 255) / 256, c->batch);
  k_env_identity<R><<<grid, 256, 0, c->stream>>>(fb, bond + 1, f.env_off[bond + 1 - f.p]);
  ++c->launches;
  return cudaGetLastError();
}

template <typename R>
cudaError_t trace_right(tnmps_ctx *c, const FitDev &f, double *ov) {
  const FitBase<R> fb = base_of<R>(c, f);
  k_env_trace<R><<<c->batch, 256, 0, c->stream>>>(fb, f.q + 1, f.env_off[f.q + 1 - f.p], ov);
  ++c->launches;
  return cudaGetLastError();
}

// <phi|G psi> over the window by left environments from the identity at bond p-1
template <typename R>
cudaError_t overlap_impl(tnmps_ctx *c, const FitDev &f, double *ov) {
  cudaError_t e;
  if ((e = boundary<R>(c, f, f.p - 1)) != cudaSuccess) return e;
  for (int i = f.p; i <= f.q; ++i)
    if ((e = env_left<R>(c, f, i, false)) != cudaSuccess) return e;
  return trace_right<R>(c, f, ov);
}

// one left-to-right sweep of two-site updates; the centre must be on p and
// phi's sites p+1..q right isometries
template <typename R>
cudaError_t sweep_impl(tnmps_ctx *c, const FitDev &f, double *ov) {
  cudaError_t e;
  cudaEvent_t ev = prof_begin(c, PC_FIT);
  if ((e = boundary<R>(c, f, f.q)) != cudaSuccess) return e;
  for (int i = f.q; i >= f.p + 2; --i)
    if ((e = env_right<R>(c, f, i)) != cudaSuccess) return e;
  if ((e = boundary<R>(c, f, f.p - 1)) != cudaSuccess) return e;
  prof_end(c, PC_FIT, ev);
  for (int i = f.p; i < f.q; ++i) {
    ev = prof_begin(c, PC_FIT);
    if ((e = pair_grad<R>(c, f, i)) != cudaSuccess) return e;
    prof_end(c, PC_FIT, ev);
    if ((e = launch_split_theta(c, i)) != cudaSuccess) return e;
    ev = prof_begin(c, PC_FIT);
    if ((e = env_left<R>(c, f, i, true)) != cudaSuccess) return e;  // T2 of this pair
    prof_end(c, PC_FIT, ev);
  }
  ev = prof_begin(c, PC_FIT);
  if ((e = env_left<R>(c, f, f.q, false)) != cudaSuccess) return e;
  if ((e = trace_right<R>(c, f, ov)) != cudaSuccess) return e;
  prof_end(c, PC_FIT, ev);
  return cudaSuccess;
}

}  // namespace

cudaError_t fit_overlap(tnmps_ctx *c, const FitDev &f, double *ov) {
  return c->dtype == TNMPS_C128 ? overlap_impl<double>(c, f, ov) : overlap_impl<float>(c, f, ov);
}

cudaError_t fit_sweep(tnmps_ctx *c, const FitDev &f, double *ov) {
  return c->dtype == TNMPS_C128 ? sweep_impl<double>(c, f, ov) : sweep_impl<float>(c, f, ov);
}

cudaError_t fit_finish(tnmps_ctx *c, const double *saved, const double *ov) {
  k_fit_finish<<<(c->batch + 255) / 256, 256, 0, c->stream>>>(saved, ov, c->discarded, c->batch);
  ++c->launches;
  return cudaGetLastError();
}
