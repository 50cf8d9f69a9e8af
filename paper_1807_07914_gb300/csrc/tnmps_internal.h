// Internal declarations shared by the CUDA translation units of libtnmps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tnmps.h"

// ---------------------------------------------------------------- complex
template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> z;
  z.re = a;
  z.im = b;
  return z;
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return mkc<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mkc<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cx<R> cconj(cx<R> a) {
  return mkc<R>(a.re, -a.im);
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// ---------------------------------------------------------------- limits
#define TNMPS_MAX_CHI 256
#define TNMPS_MAX_FAC 8          // fused single-qubit factors per side of one op
#define TNMPS_MAX_MPO_BOND 64    // super-gate MPO bond cap (after compression)
#define TNMPS_JACOBI_MAX_DIM 512

// device error flag bits
#define TNMPS_EFLAG_NOT_CONVERGED 1u
#define TNMPS_EFLAG_NUMERIC 2u
#define TNMPS_EFLAG_TIMEOUT 4u

// device counter slots (uint64)
enum {
  CNT_GATES2Q = 0,
  CNT_GATES2Q_FULL,
  CNT_PAIR_ROWS,
  CNT_ROTATIONS,
  CNT_SWEEPS,
  CNT_SVDS,
  CNT_ENV_UPDATES,
  CNT_ENV_FLOPS,
  CNT_ROT_ROWS,
  CNT_JAC_BYTES,
  CNT_NUM
};

// kernel classes for event timing (mirrors tnmps_prof_class in tnmps.h)
enum {
  PC_THETA = 0, PC_JACOBI, PC_SPLIT, PC_MOVE, PC_GATE1, PC_ENV, PC_TERM, PC_ENV_TC, PC_FIT,
  PC_SVD_LQ, PC_NUM
};

// ---------------------------------------------------------------- ops
// A single-qubit factor: fixed 2x2 (kind 0, row-major complex in m[]) or a
// parameterised rotation (kind 1/2/3 = RX/RY/RZ) of angle
// angle + scale * theta[param] (param < 0: angle alone).
struct Fac1 {
  int32_t kind, param;
  double angle, scale;
  double m[8];
};

// Fused two-qubit op on sites (l, l+1): G = core * (U_l (x) U_{l+1}), where
// U_s = f_{k-1} ... f_1 f_0 of the side's factor list; core is a fixed 4x4
// (row-major complex, basis 2*s_l + s_{l+1}).
struct Op2 {
  int32_t l, nl, nr, pad;
  double core[32];
  Fac1 fl[TNMPS_MAX_FAC];
  Fac1 fr[TNMPS_MAX_FAC];
};

// Standalone single-qubit op on one site.
struct Op1 {
  int32_t site, nf, pad0, pad1;
  Fac1 f[TNMPS_MAX_FAC];
};

// A planned op: fused two-qubit gate or standalone single-qubit op.
struct PlannedOp {
  bool two;
  Op2 o2;
  Op1 o1;
};
// Validate a gate list for an n-qubit register, expand distant two-qubit
// gates into SWAP chains and fuse single-qubit runs into the next two-qubit
// op on their site. On failure *err describes the problem.
tnmps_status plan_gates(int n, const tnmps_gate *gates, size_t n_gates, size_t n_params,
                        std::vector<PlannedOp> &out, std::string &err);

// ---------------------------------------------------------------- layout
// Device view of the batched MPS, passed by value to kernels.
struct StateView {
  void *sites;            // complex elements, state b at sites + b*state_elems
  const int64_t *site_off;  // device: element offset of each site in a state
  int32_t *dims;          // [batch][n+1]: dims[b][i] = D_{i-1}; D_{-1} = D_{n-1} = 1
  int64_t state_elems;
  int32_t n, batch, chi;
};

struct tnmps_ctx {
  int n = 0, chi = 0, batch = 0, max_params = 0;
  tnmps_dtype dtype = TNMPS_C128;
  double eps = 1e-4;
  float jacobi_tolfac = 1.0f;     // factor on the Jacobi orthogonality tolerance
  int svd_lq = 1;                 // 1: Jacobi on L of Theta = L Q^H (0: on Theta)
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;

  // carved device regions
  void *sites = nullptr;
  int64_t *site_off_dev = nullptr;
  int32_t *dims = nullptr;
  void *theta_buf = nullptr;   // [batch][tw] row-major Theta (gate applied)
  void *w_buf = nullptr;       // [batch][tw] column-major Jacobi working copy
  void *q_buf = nullptr;       // [batch][tw] Householder scratch of the block's LQ
  double *sigma = nullptr;     // [batch][2chi]
  int32_t *perm = nullptr;     // [batch][2chi]
  double *scale = nullptr;     // [batch]
  double *discarded = nullptr; // [batch]
  double *theta_dev = nullptr; // [batch][max_params]
  uint32_t *err = nullptr;     // device flags
  unsigned long long *counters = nullptr;  // [CNT_NUM]
  void *ebuf = nullptr;        // [batch][chi^2] complex128 Gram (complex64 form)
  void *tc_a = nullptr;        // BF16-split form: [batch] converted K2 operands (C_l)
  void *tc_b = nullptr;        //                  [batch] converted K2 operands (B_{l+1}^T)
  int64_t tc_a_stride = 0, tc_b_stride = 0;

  // instrumentation: host-side launch count and optional per-class event timing
  uint64_t launches = 0;
  uint32_t prof_mask = 0;
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_open;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[PC_NUM] = {0};
  uint64_t prof_cnt[PC_NUM] = {0};

  std::vector<int64_t> site_off;  // host copy
  std::vector<int> cap;           // bond capacity, size n+1 (cap[0] = cap[n] = 1)
  int64_t state_elems = 0;
  int64_t tw = 0;                 // (2 chi)^2

  // host-side planning state; centre -1 = product state (any site may be the centre)
  int centre = -1;
  int fit_cap = 0;                // > 0: extra bond cap of the splits (super-gate fit stages)
  std::vector<int> ub;            // upper bound of dims per bond index 0..n
  std::string last_error;
  int inject_nth = 0;
  tnmps_status inject_status = TNMPS_OK;
  int call_count = 0;

  uint64_t uid = 0;               // unique per tnmps_init in this process (never reused)
  tnmps_tuning tuning{};          // launch shapes (all zero: defaults)

  // last uploaded term plan (skip re-upload)
  const void *plan_terms = nullptr;
  void *plan_ws = nullptr;
  uint64_t plan_gen = 0;

  StateView view() const {
    StateView v;
    v.sites = sites;
    v.site_off = site_off_dev;
    v.dims = dims;
    v.state_elems = state_elems;
    v.n = n;
    v.batch = batch;
    v.chi = chi;
    return v;
  }
};

// ---------------------------------------------------------------- timing
inline cudaEvent_t prof_event(tnmps_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
inline cudaEvent_t prof_begin(tnmps_ctx *c, int cls) {
  if (!(c->prof_mask & (1u << cls))) return nullptr;
  cudaEvent_t a = prof_event(c);
  cudaEventRecord(a, c->stream);
  return a;
}
inline void prof_end(tnmps_ctx *c, int cls, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b = prof_event(c);
  cudaEventRecord(b, c->stream);
  c->prof_open.push_back({cls, a, b});
}

// ---------------------------------------------------------------- launchers
// Each returns cudaSuccess or the launch error. dtype dispatch inside.
cudaError_t launch_init_state(tnmps_ctx *c);
cudaError_t launch_gate2(tnmps_ctx *c, const Op2 &op, const double *theta, int64_t th_stride);
cudaError_t launch_gate1(tnmps_ctx *c, const Op1 &op, const double *theta, int64_t th_stride);
// K3 + K4 on the block already in theta_buf (identity gate): rank under the
// bond cap, A_l <- U_k, C_{l+1} <- U_k^H Theta normalised; centre to l+1
cudaError_t launch_split_theta(tnmps_ctx *c, int l);
cudaError_t launch_move_right(tnmps_ctx *c, int site);
cudaError_t launch_move_left(tnmps_ctx *c, int site);
// Measurement shots (centre on site n-1): u [batch][shots][n] -> bits
cudaError_t launch_sample(tnmps_ctx *c, const double *u, int shots, uint8_t *bits);
// K2 of the BF16-split form: Theta = C_l B_{l+1} on the tensor cores into
// theta_buf (row-major, 2D_{l-1} x 2D_{l+1}); bytes per state of its operands
cudaError_t launch_theta_tc(tnmps_ctx *c, int l);
int64_t theta_tc_a_bytes(int chi);
int64_t theta_tc_b_bytes(int chi);
// K4 of the BF16-split form: C_{l+1} = U_k^H Theta on the tensor cores into site
// l+1 (U_k in site l, Theta in theta_buf, k = dims[l+1] <= kub)
cudaError_t launch_split_tc(tnmps_ctx *c, int l, int kub);
cudaError_t launch_jacobi_standalone(tnmps_dtype dt, int batch, int m, int n, void *a, int lda,
                                     double *sigma, int32_t *sweeps, int max_sweeps,
                                     cudaStream_t s);

// Super-gate fit over the window [p, q] (device buffers carved from the
// caller's workspace; element counts in the context's complex type).
struct FitDev {
  int p = 0, q = 0;
  const void *psi = nullptr;      // snapshot of psi's window sites, per state psi_stride
  int64_t psi_stride = 0, psi_base = 0;  // psi_base = site_off[p]
  const int32_t *pdims = nullptr; // [batch][n+1] psi dims
  void *s1 = nullptr, *s2 = nullptr, *s3 = nullptr;  // scratch, per state s_stride
  int64_t s_stride = 0;
  void *env = nullptr;            // environment slots of bonds p-1..q, per state env_stride
  int64_t env_stride = 0;
  const void *mpo = nullptr;      // MPO tensors [w_{i-1}][2][2][w_i], sites p..q
  std::vector<int64_t> mpo_off;   // per window site
  std::vector<int> w;             // MPO bonds, w[0] = w[q-p+1] = 1
  std::vector<int64_t> env_off;   // per bond p-1..q
  std::vector<int> pub;           // upper bounds of psi dims, size n+1
};
// <phi|G psi> over the window into ov[batch][2] (FP64 re, im)
cudaError_t fit_overlap(tnmps_ctx *c, const FitDev &f, double *ov);
// one left-to-right sweep of two-site updates (centre on p before, on q
// after); ov receives <phi|G psi> after the sweep
cudaError_t fit_sweep(tnmps_ctx *c, const FitDev &f, double *ov);
// discarded = saved + max(0, 1 - |ov|^2)
cudaError_t fit_finish(tnmps_ctx *c, const double *saved, const double *ov);

// expectation plan (built on the host)
struct TermPlan {
  int n = 0;
  int64_t n_terms = 0;
  int32_t depth = 0;
  // trie nodes grouped by level; node ids are level-local
  std::vector<int64_t> level_start;   // size depth+1: offsets into node arrays
  std::vector<int32_t> node_site;     // site of each node
  std::vector<int32_t> node_parent;   // parent index within previous level, -1 = identity start
  std::vector<uint8_t> node_pauli;    // Pauli applied at node_site (0..3)
  // terms attached per level: (term index, node index within level)
  std::vector<int64_t> tlevel_start;  // size depth+1
  std::vector<int32_t> tterm;
  std::vector<int32_t> tnode;
  std::vector<int32_t> tsite;         // end site b of the term
  std::vector<int32_t> identity_terms;
  std::vector<double> coeffs;
  int64_t max_level_nodes = 0;
  int64_t max_level_terms = 0;
};

cudaError_t expect_run(tnmps_ctx *c, const TermPlan &p, char *ws, size_t ws_bytes, int chunk,
                       double *energy_dev, double *per_term_dev, double **energy_used,
                       double **per_term_used);
// Workspace bytes of an expectation call; the per-term / energy result regions
// are counted only when requested (the caller then supplies no device output).
// failure-detection test kernel (k_diag.cu): a bounded wait that runs out
cudaError_t launch_debug_wait(uint32_t *err, int64_t max_cycles, cudaStream_t s);

size_t expect_ws_bytes(const tnmps_ctx *c, const TermPlan &p, int chunk, bool pt_region = true,
                       bool e_region = true);
tnmps_status expect_noalloc_impl(tnmps_ctx *c, const TermPlan &p, uint64_t gen,
                                 double *energy_dev, double *per_term_dev);
