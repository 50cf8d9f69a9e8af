// K9: hundreds of independent circuits -- uneven qubit counts, depths, bond
// caps and Pauli sums -- in one persistent launch (complex64 state, FP64
// energies).
//
// Each CTA pulls whole jobs from an atomic work counter over a host-sorted
// order (most expensive first, so the tail stays short) and runs the job end
// to end in its own scratch slice: product-state init, the planned op stream
// of the job (fused two-qubit gates with the one-sided Jacobi SVD, standalone
// single-qubit ops, QR/LQ gauge moves, all through the same CTA-level
// building blocks as the batched kernels), then the right environments and a
// depth-first walk of the job's Pauli-term trie with an environment stack,
// accumulating E = sum_k c_k <P_k> in FP64 in a fixed order.
#include <math.h>

#include <algorithm>
#include <map>
#include <new>

#include "gate_dev.cuh"
#include "gates_dev.cuh"
#include "gemm_tile.cuh"
#include "jacobi_dev.cuh"
#include "tnmps_internal.h"

#define BATCH_MAX_N 256

namespace {

struct BJob {
  int32_t n, chi, n_ops, op0, theta0, node0, n_nodes, depth;
  double e_const;
};
enum { BOP_GATE2 = 0, BOP_GATE1 = 1, BOP_RIGHT = 2, BOP_LEFT = 3 };
struct BOp {
  int32_t type, site, nl, nr, fac0, core;
};
struct BNode {
  int32_t site, pauli, depth, pad;
  double coeff;  // summed coefficients of the terms ending at this node
};

struct BatchArgs {
  const BJob *jobs;
  const int32_t *order;
  int n_jobs;
  const BOp *ops;
  const Fac1 *facs;
  const double *cores;
  const double *thetas;
  const BNode *nodes;
  double *energy, *discarded;
  int *counter;
  uint32_t *err;
  char *scratch;
  int64_t stride;  // scratch bytes per CTA
  int64_t o_state, o_t, o_w, o_e, o_renv, o_env, o_tm, o_q;
  int chi_cap;
  double eps_eff;
};

__device__ __forceinline__ int capof(int i, int n, int chi) {
  if (i <= 0 || i >= n) return 1;
  const int e = i < n - i ? i : n - i;
  return e >= 30 ? chi : min(chi, 1 << e);
}

// Generic complex GEMM operands: element (i, k) of A at A[i*ars + k*acs],
// optionally conjugated, zero below the diagonal (k < i), or with a Pauli
// acting on the k index (k = 2a + s: reads s ^ flip, phase of P).
template <typename R, bool AK, bool BK>
struct GP {
  const cx<R> *A;
  int64_t ars, acs;
  int aconj, atri, apauli;
  const cx<R> *B;
  int64_t brs, bcs;
  int bconj, btri;
  cx<R> *C;
  int64_t crs;
  static constexpr bool A_KFAST = AK, B_KFAST = BK;
  __device__ cx<R> a(int i, int k) const {
    if (atri && k < i) return mkc<R>(0, 0);
    const int flip = (apauli == 1 || apauli == 2) ? 1 : 0;
    cx<R> x = A[(int64_t)i * ars + (int64_t)(k ^ flip) * acs];
    if (apauli == 2) x = (k & 1) ? mkc<R>(-x.im, x.re) : mkc<R>(x.im, -x.re);
    else if (apauli == 3 && (k & 1)) x = mkc<R>(-x.re, -x.im);
    return aconj ? cconj(x) : x;
  }
  __device__ cx<R> b(int k, int j) const {
    if (btri && k < j) return mkc<R>(0, 0);
    const cx<R> x = B[(int64_t)k * brs + (int64_t)j * bcs];
    return bconj ? cconj(x) : x;
  }
  __device__ void store(int i, int j, cx<R> v) const { C[(int64_t)i * crs + j] = v; }
};

template <typename R, class P>
__device__ void cta_gemm(const P &p, int M, int N, int K, bool upper = false) {
  constexpr int BM = GemmCfg<R>::BM, BN = GemmCfg<R>::BN;
  P q = p;
  for (int i0 = 0; i0 < M; i0 += BM)
    for (int j0 = 0; j0 < N; j0 += BN)
      if (!upper || i0 / BM <= j0 / BN) gemm_tile<R>(q, M, N, K, i0, j0);
  __syncthreads();
}

// same, accumulating in FP32 within each K slice and in FP64 across slices
template <class P>
__device__ void cta_gemm_mixed(const P &p, int M, int N, int K, bool upper = false) {
  constexpr int BM = GemmCfg<float>::BM, BN = GemmCfg<float>::BN;
  P q = p;
  for (int i0 = 0; i0 < M; i0 += BM)
    for (int j0 = 0; j0 < N; j0 += BN)
      if (!upper || i0 / BM <= j0 / BN) gemm_tile_mixed(q, M, N, K, i0, j0);
  __syncthreads();
}

// E = U^H U - I (FP64 result, FP32 slice sums added in FP64), mirrored upper tiles
struct GramP {
  const cx<float> *U;
  cx<double> *E;
  int k;
  static constexpr bool A_KFAST = false, B_KFAST = false;
  __device__ cx<float> a(int q, int i) const { return cconj(U[(int64_t)i * k + q]); }
  __device__ cx<float> b(int i, int q) const { return U[(int64_t)i * k + q]; }
  // one writer per entry pair (upper triangle); the diagonal is real
  __device__ void store(int q, int r, cx<double> v) const {
    if (q > r) return;
    if (q == r) {
      E[(int64_t)q * k + q] = mkc<double>(v.re - 1.0, 0.0);
      return;
    }
    E[(int64_t)q * k + r] = v;
    E[(int64_t)r * k + q] = cconj(v);
  }
};
struct OrthoP {
  const cx<float> *U;
  const cx<double> *E;
  cx<float> *O;
  int k;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ cx<float> a(int i, int q) const { return U[(int64_t)i * k + q]; }
  __device__ cx<float> b(int q, int r) const {
    const cx<double> e = E[(int64_t)q * k + r];
    return mkc<float>((float)((q == r ? 1.0 : 0.0) - 0.5 * e.re), (float)(-0.5 * e.im));
  }
  __device__ void store(int i, int r, cx<float> v) const { O[(int64_t)i * k + r] = v; }
};

template <typename R>
__device__ void cta_copy(cx<R> *dst, const cx<R> *src, int64_t n) {
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
  __syncthreads();
}

template <int BC>
__global__ void __launch_bounds__(256, 1) k_batch(BatchArgs a) {
  using R = float;
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *S0 = reinterpret_cast<cx<R> *>(smraw);
  cx<R> *S1 = S0 + BC * 256;
  // third Jacobi staging slot (next block copied ahead) where it fits beside the
  // kernel's static shared memory: 16-column blocks only
  cx<R> *S2 = BC == 16 ? S1 + BC * 256 : nullptr;
  __shared__ int64_t s_off[BATCH_MAX_N + 1];
  __shared__ int64_t s_roff[BATCH_MAX_N + 1];
  __shared__ int s_dims[BATCH_MAX_N + 1];
  __shared__ int s_job;
  __shared__ cx<R> G[16];
  __shared__ double s_red[8];
  char *base = a.scratch + (int64_t)blockIdx.x * a.stride;
  cx<R> *st = reinterpret_cast<cx<R> *>(base + a.o_state);
  cx<R> *T = reinterpret_cast<cx<R> *>(base + a.o_t);
  cx<R> *W = reinterpret_cast<cx<R> *>(base + a.o_w);
  cx<double> *Eb = reinterpret_cast<cx<double> *>(base + a.o_e);
  cx<R> *renv = reinterpret_cast<cx<R> *>(base + a.o_renv);
  cx<R> *envs = reinterpret_cast<cx<R> *>(base + a.o_env);
  cx<R> *Tm = reinterpret_cast<cx<R> *>(base + a.o_tm);
  cx<R> *Qs = reinterpret_cast<cx<R> *>(base + a.o_q);  // Householder scratch of the LQ
  const int64_t env_elems = (int64_t)a.chi_cap * a.chi_cap;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_job = atomicAdd(a.counter, 1);
    __syncthreads();
    const int jj = s_job;
    __syncthreads();
    if (jj >= a.n_jobs) break;
    const int job = a.order[jj];
    const BJob J = a.jobs[job];
    const int n = J.n, chi = J.chi;
    const double *theta = a.thetas + J.theta0;
    if (tid == 0) {
      int64_t o = 0, ro = 0;
      for (int i = 0; i < n; ++i) {
        s_off[i] = o;
        o += (int64_t)capof(i, n, chi) * 2 * capof(i + 1, n, chi);
        o = (o + 31) & ~(int64_t)31;
        s_roff[i] = ro;
        ro += (int64_t)capof(i + 1, n, chi) * capof(i + 1, n, chi);
      }
    }
    for (int i = tid; i <= n; i += blockDim.x) s_dims[i] = 1;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      st[s_off[i]] = mkc<R>(1, 0);  // |0> on every site
      st[s_off[i] + 1] = mkc<R>(0, 0);
    }
    __syncthreads();
    double discarded = 0;
    bool fail = false;

    for (int t = 0; t < J.n_ops && !fail; ++t) {
      const BOp op = a.ops[J.op0 + t];
      if (op.type == BOP_GATE2) {
        const int l = op.site;
        const int Dl = s_dims[l], Dm = s_dims[l + 1], Dr = s_dims[l + 2];
        const int M = 2 * Dl, N = 2 * Dr;
        cx<R> *Cl = st + s_off[l], *Bn = st + s_off[l + 1];
        GP<R, true, false> px{Cl, Dm, 1, 0, 0, 0, Bn, N, 1, 0, 0, T, N};
        cta_gemm<R>(px, M, N, Dm);
        if (tid == 0) {
          cx<double> Gd[16];
          op2_matrix_parts(a.cores + 32 * op.core, a.facs + op.fac0, op.nl,
                           a.facs + op.fac0 + op.nl, op.nr, theta, Gd);
          for (int e = 0; e < 16; ++e) G[e] = mkc<R>((R)Gd[e].re, (R)Gd[e].im);
        }
        __syncthreads();
        gdev::apply_gate4_range<R>(G, T, nullptr, Dl, Dr, tid, blockDim.x);
        __syncthreads();
        // Theta = L Q^H: the Jacobi runs on L (same singular values and left
        // vectors, fewer sweeps); its columns past min(M, N) are zero
        const int r = gdev::lq_theta_cta<R, 8>(T, M, N, Qs, W);
        bool conv;
        int rot, chk;
        // 8 warps: with 16-column blocks each warp keeps its two x columns in registers
        jac::jacobi_run<R, BC, 8, BC == 16, BC == 16>(W, M, r, M, S0, S1, 1.0f, 30, &conv, &rot,
                                                      &chk, S2);
        if (!conv && N > 1) {
          if (tid == 0) atomicOr(a.err, TNMPS_EFLAG_NOT_CONVERGED);
        }
        double w;
        bool bad;
        const int k = gdev::select_cta<R>(W, M, N, capof(l + 1, n, chi), a.eps_eff, Cl, &w, &bad);
        if (bad) {
          if (tid == 0) atomicOr(a.err, TNMPS_EFLAG_NUMERIC);
          fail = true;
          break;
        }
        discarded += w;
        // re-orthonormalise U_k with the FP64 Gram: U <- U (I - E/2)
        GramP pg{Cl, Eb, k};
        cta_gemm_mixed(pg, k, k, M, true);
        OrthoP po{Cl, Eb, W, k};
        cta_gemm<R>(po, M, k, k);
        cta_copy<R>(Cl, W, (int64_t)M * k);
        // C_{l+1} = U_k^H Theta, renormalised
        GP<R, false, false> ps{Cl, 1, k, 1, 0, 0, T, N, 1, 0, 0, Bn, N};
        cta_gemm<R>(ps, k, N, M);
        if (tid == 0) s_dims[l + 1] = k;
        __syncthreads();
        gdev::normalise_cta<R>(Bn, k * N);
      } else if (op.type == BOP_GATE1) {
        if (tid == 0) {
          cx<double> Ud[4];
          side_matrix(a.facs + op.fac0, op.nl, theta, Ud);
          for (int e = 0; e < 4; ++e) G[e] = mkc<R>((R)Ud[e].re, (R)Ud[e].im);
        }
        __syncthreads();
        const int Dl = s_dims[op.site], Dr = s_dims[op.site + 1];
        cx<R> *X = st + s_off[op.site];
        for (int e = tid; e < Dl * Dr; e += blockDim.x) {
          const int aa = e / Dr, c = e - aa * Dr;
          const cx<R> x0 = X[(int64_t)(2 * aa) * Dr + c], x1 = X[(int64_t)(2 * aa + 1) * Dr + c];
          cx<R> y0 = mkc<R>(0, 0), y1 = mkc<R>(0, 0);
          cfma(y0, G[0], x0);
          cfma(y0, G[1], x1);
          cfma(y1, G[2], x0);
          cfma(y1, G[3], x1);
          X[(int64_t)(2 * aa) * Dr + c] = y0;
          X[(int64_t)(2 * aa + 1) * Dr + c] = y1;
        }
        __syncthreads();
      } else if (op.type == BOP_RIGHT) {
        const int c = op.site;
        const int Dl = s_dims[c], Dr = s_dims[c + 1], N2 = 2 * s_dims[c + 2];
        const int r = gdev::qr_right_cta<R>(st + s_off[c], Dl, Dr, W, T);
        // R (upper triangle of W, ld 2Dl) times B_{c+1}
        GP<R, false, false> p{W, 1, 2 * Dl, 0, 1, 0, st + s_off[c + 1], N2, 1, 0, 0, T, N2};
        cta_gemm<R>(p, r, N2, Dr);
        cta_copy<R>(st + s_off[c + 1], T, (int64_t)r * N2);
        if (tid == 0) s_dims[c + 1] = r;
        __syncthreads();
      } else {  // BOP_LEFT
        const int c = op.site;
        const int Dl = s_dims[c], Dr = s_dims[c + 1], D0 = s_dims[c - 1];
        const int r = gdev::lq_left_cta<R>(st + s_off[c], Dl, Dr, W, T);
        // A_{c-1} times L = R'^H (R' upper triangle of W, ld 2Dr)
        GP<R, true, false> p{st + s_off[c - 1], Dl, 1, 0, 0, 0, W, 2 * Dr, 1, 1, 1, T, r};
        cta_gemm<R>(p, 2 * D0, r, Dl);
        cta_copy<R>(st + s_off[c - 1], T, (int64_t)2 * D0 * r);
        if (tid == 0) s_dims[c] = r;
        __syncthreads();
      }
    }
    if (fail) {
      if (tid == 0) a.energy[job] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }

    // right environments R_i (sites i+1..n-1, identity), R_{n-1} = 1
    if (tid == 0) renv[s_roff[n - 1]] = mkc<R>(1, 0);
    __syncthreads();
    for (int i = n - 2; i >= 0; --i) {
      const int Dl = s_dims[i + 1], Dr = s_dims[i + 2];
      const cx<R> *X = st + s_off[i + 1];
      GP<R, true, true> py{X, Dr, 1, 0, 0, 0, renv + s_roff[i + 1], 1, Dr, 0, 0, Tm, Dr};
      cta_gemm<R>(py, 2 * Dl, Dr, Dr);
      GP<R, true, true> pr{X, 2 * Dr, 1, 1, 0, 0, Tm, 1, 2 * Dr, 0, 0, renv + s_roff[i], Dl};
      cta_gemm<R>(pr, Dl, Dl, 2 * Dr);
    }
    // depth-first walk of the trie: env[d-1] holds the node at depth d
    double E = J.e_const;
    for (int v = 0; v < J.n_nodes; ++v) {
      const BNode nd = a.nodes[J.node0 + v];
      const int s = nd.site, d = nd.depth;
      const int Dl = s_dims[s], Dr = s_dims[s + 1];
      const cx<R> *X = st + s_off[s];
      cx<R> *out = envs + (int64_t)(d - 1) * env_elems;
      const cx<R> *src = X;
      if (d > 1) {
        GP<R, true, false> p1{envs + (int64_t)(d - 2) * env_elems, Dl, 1, 0, 0, 0, X, 2 * Dr,
                              1, 0, 0, Tm, 2 * Dr};
        cta_gemm<R>(p1, Dl, 2 * Dr, Dl);
        src = Tm;
      }
      GP<R, false, false> p2{X, 1, Dr, 1, 0, nd.pauli, src, Dr, 1, 0, 0, out, Dr};
      cta_gemm<R>(p2, Dr, Dr, 2 * Dl);
      if (nd.coeff != 0.0) {
        const cx<R> *Rr = renv + s_roff[s];
        double acc = 0;
        for (int e = tid; e < Dr * Dr; e += blockDim.x)
          acc += (double)out[e].re * Rr[e].re - (double)out[e].im * Rr[e].im;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
          double tot = 0;
          for (int w = 0; w < 8; ++w) tot += s_red[w];
          E += nd.coeff * tot;
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      a.energy[job] = E;
      a.discarded[job] = discarded;
      if (!isfinite(E)) atomicOr(a.err, TNMPS_EFLAG_NUMERIC);
    }
  }
}

}  // namespace

// ====================================================================== host
struct tnmps_batch {
  int n_jobs = 0, chi_cap = 0, n_max = 0, depth_max = 0;
  double cutoff = 1e-4;
  std::vector<BJob> jobs;
  std::vector<int32_t> order;
  std::vector<BOp> ops;
  std::vector<Fac1> facs;
  std::vector<double> cores, thetas;
  std::vector<BNode> nodes;
  std::vector<double> cost;
  int64_t state_max = 0, renv_max = 0;
  // device binding
  char *arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t stream = nullptr;
  BatchArgs args{};
  int grid = 0, bc = 32;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;  // private stream for graph capture
  std::string last_error;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t state_elems(int n, int chi) {
  int64_t o = 0;
  for (int i = 0; i < n; ++i) {
    auto cap = [&](int k) -> int64_t {
      if (k <= 0 || k >= n) return 1;
      const int e = std::min(k, n - k);
      return e >= 30 ? chi : std::min(chi, 1 << e);
    };
    o += cap(i) * 2 * cap(i + 1);
    o = (o + 31) & ~(int64_t)31;
  }
  return o;
}

struct Sizes {
  int64_t o_state, o_t, o_w, o_e, o_renv, o_env, o_tm, o_q, stride;
  size_t plan_bytes, total;
  size_t o_jobs, o_order, o_ops, o_facs, o_cores, o_thetas, o_nodes, o_energy, o_disc, o_counter,
      o_err, o_scratch;
};

Sizes sizes(const tnmps_batch *b, int grid) {
  Sizes s{};
  const int64_t c2 = (int64_t)b->chi_cap * b->chi_cap;
  int64_t o = 0;
  auto put = [&](int64_t bytes) {
    const int64_t at = o;
    o = (int64_t)al256((size_t)(o + bytes));
    return at;
  };
  s.o_state = put(8 * b->state_max);
  s.o_t = put(8 * 4 * c2);
  s.o_w = put(8 * 4 * c2);
  s.o_e = put(16 * c2);
  s.o_renv = put(8 * b->renv_max);
  s.o_env = put(8 * c2 * std::max(b->depth_max, 1));
  s.o_tm = put(8 * 2 * c2);
  s.o_q = put(8 * 4 * c2);
  s.stride = o;
  size_t p = 0;
  auto plan = [&](size_t bytes) {
    const size_t at = p;
    p = al256(p + bytes);
    return at;
  };
  s.o_jobs = plan(sizeof(BJob) * b->jobs.size());
  s.o_order = plan(4 * b->order.size());
  s.o_ops = plan(sizeof(BOp) * std::max<size_t>(b->ops.size(), 1));
  s.o_facs = plan(sizeof(Fac1) * std::max<size_t>(b->facs.size(), 1));
  s.o_cores = plan(8 * std::max<size_t>(b->cores.size(), 1));
  s.o_thetas = plan(8 * std::max<size_t>(b->thetas.size(), 1));
  s.o_nodes = plan(sizeof(BNode) * std::max<size_t>(b->nodes.size(), 1));
  s.o_energy = plan(8 * b->jobs.size());
  s.o_disc = plan(8 * b->jobs.size());
  s.o_counter = plan(4);
  s.o_err = plan(4);
  s.plan_bytes = p;
  s.o_scratch = p;
  s.total = p + (size_t)grid * (size_t)s.stride;
  return s;
}

// depth-first preorder of one job's term trie with summed coefficients
void build_trie(int n, const int32_t *off, const int32_t *sites, const uint8_t *paulis,
                const double *coeffs, int T, std::vector<BNode> &out, double &e_const,
                int &depth, std::string &err, bool &ok) {
  struct Nd {
    int site, pauli, depth;
    double coeff;
    std::vector<int> kids;
  };
  std::vector<Nd> nd;
  std::map<std::pair<long, int>, int> child;
  std::vector<int> roots;
  std::vector<int> ops(n);
  e_const = 0;
  ok = true;
  for (int k = 0; k < T; ++k) {
    if (off[k] == off[k + 1]) {
      e_const += coeffs[k];
      continue;
    }
    std::fill(ops.begin(), ops.end(), 0);
    int lo = n, hi = -1;
    for (int j = off[k]; j < off[k + 1]; ++j) {
      const int s = sites[j], q = paulis[j];
      if (s < 0 || s >= n || q < 1 || q > 3 || ops[s]) {
        err = "invalid Pauli term";
        ok = false;
        return;
      }
      ops[s] = q;
      lo = std::min(lo, s);
      hi = std::max(hi, s);
    }
    long cur = -1 - (long)lo;
    for (int s = lo; s <= hi; ++s) {
      auto key = std::make_pair(cur, ops[s]);
      auto it = child.find(key);
      if (it == child.end()) {
        nd.push_back({s, ops[s], s - lo + 1, 0.0, {}});
        const int id = (int)nd.size() - 1;
        if (cur >= 0) nd[cur].kids.push_back(id);
        else roots.push_back(id);
        it = child.emplace(key, id).first;
      }
      cur = it->second;
    }
    nd[cur].coeff += coeffs[k];
  }
  depth = 0;
  std::vector<int> stack(roots.rbegin(), roots.rend());
  while (!stack.empty()) {
    const int v = stack.back();
    stack.pop_back();
    out.push_back({nd[v].site, nd[v].pauli, nd[v].depth, 0, nd[v].coeff});
    depth = std::max(depth, nd[v].depth);
    for (auto it = nd[v].kids.rbegin(); it != nd[v].kids.rend(); ++it) stack.push_back(*it);
  }
}

}  // namespace

extern "C" {

tnmps_status tnmps_batch_create(tnmps_batch **out, const tnmps_job *jobs, int n_jobs,
                                double cutoff) {
  if (!out || !jobs || n_jobs < 1 || !(cutoff >= 0)) return TNMPS_ERR_ARG;
  *out = nullptr;
  tnmps_batch *b = new (std::nothrow) tnmps_batch();
  if (!b) return TNMPS_ERR_NOMEM;
  b->n_jobs = n_jobs;
  b->cutoff = cutoff;
  std::map<std::vector<double>, int> core_ids;
  for (int j = 0; j < n_jobs; ++j) {
    const tnmps_job &jb = jobs[j];
    if (jb.n_qubits < 2 || jb.n_qubits > BATCH_MAX_N || jb.chi_max < 1 ||
        jb.chi_max > 128 || jb.n_params < 0 || (jb.n_params && !jb.theta)) {
      delete b;
      return TNMPS_ERR_ARG;
    }
    std::vector<PlannedOp> planned;
    std::string err;
    tnmps_status st = plan_gates(jb.n_qubits, jb.gates, (size_t)jb.n_gates, (size_t)jb.n_params,
                                 planned, err);
    if (st != TNMPS_OK) {
      delete b;
      return st;
    }
    BJob J{};
    J.n = jb.n_qubits;
    J.chi = jb.chi_max;
    J.op0 = (int32_t)b->ops.size();
    J.theta0 = (int32_t)b->thetas.size();
    b->thetas.insert(b->thetas.end(), jb.theta, jb.theta + jb.n_params);
    // gauge moves exactly as the single-context planner schedules them
    int centre = -1;
    std::vector<int> ub(J.n + 1, 1);
    auto cap = [&](int k) {
      if (k <= 0 || k >= J.n) return 1;
      const int e = std::min(k, J.n - k);
      return e >= 30 ? J.chi : std::min(J.chi, 1 << e);
    };
    double cost = 0;
    auto move_to = [&](int target) {
      if (centre < 0) {
        centre = target;
        return;
      }
      while (centre < target) {
        b->ops.push_back({BOP_RIGHT, centre, 0, 0, 0, 0});
        cost += 4.0 * ub[centre] * ub[centre + 1] * ub[centre + 1];
        ub[centre + 1] = std::min(2 * ub[centre], ub[centre + 1]);
        ++centre;
      }
      while (centre > target) {
        b->ops.push_back({BOP_LEFT, centre, 0, 0, 0, 0});
        cost += 4.0 * ub[centre] * ub[centre] * ub[centre + 1];
        ub[centre] = std::min(2 * ub[centre + 1], ub[centre]);
        --centre;
      }
    };
    for (const PlannedOp &po : planned) {
      if (po.two) {
        move_to(po.o2.l);
        BOp o{BOP_GATE2, po.o2.l, po.o2.nl, po.o2.nr, (int32_t)b->facs.size(), 0};
        for (int i = 0; i < po.o2.nl; ++i) b->facs.push_back(po.o2.fl[i]);
        for (int i = 0; i < po.o2.nr; ++i) b->facs.push_back(po.o2.fr[i]);
        std::vector<double> core(po.o2.core, po.o2.core + 32);
        auto it = core_ids.find(core);
        if (it == core_ids.end()) {
          it = core_ids.emplace(core, (int)(b->cores.size() / 32)).first;
          b->cores.insert(b->cores.end(), core.begin(), core.end());
        }
        o.core = it->second;
        b->ops.push_back(o);
        const int l = po.o2.l;
        const double Mx = 2.0 * ub[l], Nx = 2.0 * ub[l + 2];
        cost += 8.0 * Mx * Nx * Nx;  // ~ one-sided Jacobi sweeps on Theta
        ub[l + 1] = std::min({cap(l + 1), 2 * ub[l], 2 * ub[l + 2]});
        centre = l + 1;
      } else {
        BOp o{BOP_GATE1, po.o1.site, po.o1.nf, 0, (int32_t)b->facs.size(), 0};
        for (int i = 0; i < po.o1.nf; ++i) b->facs.push_back(po.o1.f[i]);
        b->ops.push_back(o);
      }
    }
    move_to(J.n - 1);
    J.n_ops = (int32_t)b->ops.size() - J.op0;
    // Pauli sum
    J.node0 = (int32_t)b->nodes.size();
    bool ok;
    std::string err2;
    int depth = 0;
    build_trie(J.n, jb.term_off, jb.sites, jb.paulis, jb.coeffs, jb.n_terms, b->nodes,
               J.e_const, depth, err2, ok);
    if (!ok) {
      delete b;
      return TNMPS_ERR_ARG;
    }
    J.n_nodes = (int32_t)b->nodes.size() - J.node0;
    J.depth = depth;
    const double chi_eff = std::min(J.chi, 1 << std::min(J.n / 2, 20));
    cost += (double)J.n_nodes * 16.0 * chi_eff * chi_eff * chi_eff + J.n * 32.0 * chi_eff *
            chi_eff * chi_eff;
    b->jobs.push_back(J);
    b->cost.push_back(cost);
    b->chi_cap = std::max(b->chi_cap, J.chi);
    b->n_max = std::max(b->n_max, J.n);
    b->depth_max = std::max(b->depth_max, depth);
    b->state_max = std::max(b->state_max, state_elems(J.n, J.chi));
    int64_t re = 0;
    for (int i = 0; i < J.n; ++i) re += (int64_t)cap(i + 1) * cap(i + 1);
    b->renv_max = std::max(b->renv_max, re);
  }
  b->order.resize(n_jobs);
  for (int j = 0; j < n_jobs; ++j) b->order[j] = j;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  *out = b;
  return TNMPS_OK;
}

size_t tnmps_batch_bytes(const tnmps_batch *b, int ctas) {
  if (!b || ctas < 1) return 0;
  return sizes(b, ctas).total;
}

static tnmps_status bfail(tnmps_batch *b, cudaError_t e, const char *where) {
  b->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return TNMPS_ERR_CUDA;
}

tnmps_status tnmps_batch_bind(tnmps_batch *b, void *arena, size_t bytes, int ctas,
                              int block_cols, void *stream) {
  if (!b || !arena || ((uintptr_t)arena & 255) || ctas < 1 ||
      (block_cols != 16 && block_cols != 32))
    return TNMPS_ERR_ARG;
  const Sizes s = sizes(b, ctas);
  if (bytes < s.total) return TNMPS_ERR_NOMEM;
  b->arena = (char *)arena;
  b->arena_bytes = bytes;
  b->stream = (cudaStream_t)stream;
  b->grid = ctas;
  b->bc = block_cols;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  char *A = b->arena;
  cudaStream_t st = b->stream;
  cudaError_t e = cudaSuccess;
  auto up = [&](size_t off, const void *src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(A + off, src, n, cudaMemcpyHostToDevice, st);
  };
  up(s.o_jobs, b->jobs.data(), sizeof(BJob) * b->jobs.size());
  up(s.o_order, b->order.data(), 4 * b->order.size());
  up(s.o_ops, b->ops.data(), sizeof(BOp) * b->ops.size());
  up(s.o_facs, b->facs.data(), sizeof(Fac1) * b->facs.size());
  up(s.o_cores, b->cores.data(), 8 * b->cores.size());
  up(s.o_thetas, b->thetas.data(), 8 * b->thetas.size());
  up(s.o_nodes, b->nodes.data(), sizeof(BNode) * b->nodes.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(A + s.o_err, 0, 4, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bfail(b, e, "batch upload");
  BatchArgs &a = b->args;
  a.jobs = (const BJob *)(A + s.o_jobs);
  a.order = (const int32_t *)(A + s.o_order);
  a.n_jobs = b->n_jobs;
  a.ops = (const BOp *)(A + s.o_ops);
  a.facs = (const Fac1 *)(A + s.o_facs);
  a.cores = (const double *)(A + s.o_cores);
  a.thetas = (const double *)(A + s.o_thetas);
  a.nodes = (const BNode *)(A + s.o_nodes);
  a.energy = (double *)(A + s.o_energy);
  a.discarded = (double *)(A + s.o_disc);
  a.counter = (int *)(A + s.o_counter);
  a.err = (uint32_t *)(A + s.o_err);
  a.scratch = A + s.o_scratch;
  a.stride = s.stride;
  a.o_state = s.o_state;
  a.o_t = s.o_t;
  a.o_w = s.o_w;
  a.o_e = s.o_e;
  a.o_renv = s.o_renv;
  a.o_env = s.o_env;
  a.o_tm = s.o_tm;
  a.o_q = s.o_q;
  a.chi_cap = b->chi_cap;
  const double floor = 8.0 * 5.9604644775390625e-08;
  a.eps_eff = b->cutoff > floor ? b->cutoff : floor;
  return TNMPS_OK;
}

static cudaError_t enqueue(tnmps_batch *b) {
  cudaError_t e = cudaMemsetAsync(b->args.counter, 0, 4, b->stream);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)(b->bc == 16 ? 3 : 2) * b->bc * 256 * sizeof(cx<float>);
  if (b->bc == 32) {
    e = cudaFuncSetAttribute(k_batch<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_batch<32><<<b->grid, 256, smem, b->stream>>>(b->args);
  } else {
    e = cudaFuncSetAttribute(k_batch<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_batch<16><<<b->grid, 256, smem, b->stream>>>(b->args);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

tnmps_status tnmps_batch_launch(tnmps_batch *b) {
  if (!b || !b->arena) return TNMPS_ERR_ARG;
  cudaError_t e = b->graph ? cudaGraphLaunch(b->graph, b->stream) : enqueue(b);
  return e == cudaSuccess ? TNMPS_OK : bfail(b, e, "batch launch");
}

tnmps_status tnmps_batch_capture_graph(tnmps_batch *b) {
  if (!b || !b->arena) return TNMPS_ERR_ARG;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  // attributes are set outside the capture
  const size_t smem = (size_t)(b->bc == 16 ? 3 : 2) * b->bc * 256 * sizeof(cx<float>);
  cudaError_t e = b->bc == 32 ? cudaFuncSetAttribute(k_batch<32>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem)
                              : cudaFuncSetAttribute(k_batch<16>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
  if (e != cudaSuccess) return bfail(b, e, "graph attributes");
  // the legacy default stream cannot be captured: capture on a private
  // stream, replay on the batch's stream
  if (!b->capture_stream) {
    e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bfail(b, e, "capture stream");
  }
  e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e, "sync before capture");
  cudaGraph_t g = nullptr;
  const cudaStream_t keep = b->stream;
  b->stream = b->capture_stream;
  e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    b->stream = keep;
    return bfail(b, e, "begin capture");
  }
  cudaError_t e2 = enqueue(b);
  e = cudaStreamEndCapture(b->stream, &g);
  b->stream = keep;
  if (e2 != cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  return e == cudaSuccess ? TNMPS_OK : bfail(b, e, "graph capture");
}

tnmps_status tnmps_batch_results(tnmps_batch *b, double *energy, double *discarded) {
  if (!b || !b->arena || !energy) return TNMPS_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(energy, b->args.energy, 8 * (size_t)b->n_jobs,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && discarded)
    e = cudaMemcpyAsync(discarded, b->args.discarded, 8 * (size_t)b->n_jobs,
                        cudaMemcpyDeviceToHost, b->stream);
  uint32_t flags = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flags, b->args.err, 4, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e, "batch results");
  if (flags & TNMPS_EFLAG_NUMERIC) {
    b->last_error = "NaN/Inf in a job";
    return TNMPS_ERR_NUMERIC;
  }
  if (flags & TNMPS_EFLAG_NOT_CONVERGED) {
    b->last_error = "a Jacobi SVD reached its sweep cap";
    return TNMPS_ERR_NOT_CONVERGED;
  }
  if (flags & TNMPS_EFLAG_TIMEOUT) {
    b->last_error = "a device-side wait ran out";
    return TNMPS_ERR_TIMEOUT;
  }
  return TNMPS_OK;
}

tnmps_status tnmps_batch_info(const tnmps_batch *b, int64_t *n_ops, int64_t *n_nodes,
                              double *est_cost) {
  if (!b) return TNMPS_ERR_ARG;
  if (n_ops) *n_ops = (int64_t)b->ops.size();
  if (n_nodes) *n_nodes = (int64_t)b->nodes.size();
  if (est_cost) {
    double t = 0;
    for (double c : b->cost) t += c;
    *est_cost = t;
  }
  return TNMPS_OK;
}

const char *tnmps_batch_last_error(const tnmps_batch *b) {
  return b ? b->last_error.c_str() : "null batch";
}

void tnmps_batch_free(tnmps_batch *b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
}

}  // extern "C"
