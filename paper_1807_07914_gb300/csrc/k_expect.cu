// K5/K6: Pauli-sum expectation values by transfer-matrix sweeps that share
// left-environment prefixes across terms, and the FP64 energy reduction.
//
// Paper: Sec. V.B evaluates every Hamiltonian measurement term on the ansatz
// state for each parameter value; the energy is sum_k c_k <P_k>.
//
// Gauge precondition: the orthogonality centre is on site n-1, so sites
// 0..n-2 are left isometries and the left environment of any identity
// prefix is the identity matrix. A term acting on sites a..b (a, b = first
// and last non-identity site) is then
//     <P> = sum_{c,c'} L_b[c,c'] R_b[c,c'],
// where L is swept from the identity at site a through b,
//     L'[c,c'] = sum_{a,s} conj((P X)[a,s,c]) (L X)[a,s,c'],
// and R_b is the right environment of sites b+1..n-1 (identity operators),
// computed once per state. Terms are organised in a trie keyed by
// (start site, Pauli word); one transfer update per trie node serves every
// term sharing that prefix. Nodes are processed level by level, batched over
// nodes and states; each update is two complex GEMMs on the tiled core.
#include <algorithm>

#include "gemm_tile.cuh"
#include "sweep_tc.h"
#include "tnmps_internal.h"

namespace {

__device__ __forceinline__ int dimv(const StateView &v, int b, int i) {
  return v.dims[(int64_t)b * (v.n + 1) + i];
}
template <typename R>
__device__ __forceinline__ const cx<R> *site_ptr(const StateView &v, int b, int i) {
  return reinterpret_cast<const cx<R> *>(v.sites) + (int64_t)b * v.state_elems + v.site_off[i];
}

struct EnvBufs {
  void *renv;          // [Bc][renv_elems]
  const int64_t *roff; // device: offset of R_i inside one state's block
  int64_t renv_elems;
  void *lprev, *lcur;  // [nodes][Bc][chi^2]
  void *tmp;           // [nodes or Bc][Bc][2 chi^2]
  int64_t env_elems, tmp_elems;
  int b0, nb;          // state chunk
};

// ---- right environments:  Y = X R^T (2Dl x Dr),  R_i = conj(X) Y^T (Dl x Dl)
template <typename R>
struct ProbRY {
  StateView v;
  EnvBufs e;
  int i;  // computing R_i from R_{i+1} and site i+1
  const cx<R> *X, *Rn;
  cx<R> *Y;
  int Dr;
  static constexpr bool A_KFAST = true, B_KFAST = true;
  __device__ bool setup(int z, int &M, int &N, int &K) {
    const int b = e.b0 + z;
    const int Dl = dimv(v, b, i + 1);
    Dr = dimv(v, b, i + 2);
    M = 2 * Dl;
    N = Dr;
    K = Dr;
    X = site_ptr<R>(v, b, i + 1);
    Rn = reinterpret_cast<const cx<R> *>(e.renv) + (int64_t)z * e.renv_elems + e.roff[i + 1];
    Y = reinterpret_cast<cx<R> *>(e.tmp) + (int64_t)z * e.tmp_elems;
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return X[(int64_t)r * Dr + k]; }
  __device__ cx<R> b(int k, int j) const { return Rn[(int64_t)j * Dr + k]; }
  __device__ void store(int r, int j, cx<R> val) const { Y[(int64_t)r * Dr + j] = val; }
};

template <typename R>
struct ProbRR {
  StateView v;
  EnvBufs e;
  int i;
  unsigned long long *counters;
  const cx<R> *X, *Y;
  cx<R> *Ro;
  int Dl, Dr;
  static constexpr bool A_KFAST = true, B_KFAST = true;
  __device__ bool setup(int z, int &M, int &N, int &K) {
    const int b = e.b0 + z;
    Dl = dimv(v, b, i + 1);
    Dr = dimv(v, b, i + 2);
    M = Dl;
    N = Dl;
    K = 2 * Dr;
    X = site_ptr<R>(v, b, i + 1);
    Y = reinterpret_cast<const cx<R> *>(e.tmp) + (int64_t)z * e.tmp_elems;
    Ro = reinterpret_cast<cx<R> *>(e.renv) + (int64_t)z * e.renv_elems + e.roff[i];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      atomicAdd(&counters[CNT_ENV_UPDATES], 1ull);
      atomicAdd(&counters[CNT_ENV_FLOPS],
                16ull * Dl * Dr * (unsigned long long)(Dl + Dr));
    }
    return true;
  }
  __device__ cx<R> a(int r, int k) const { return cconj(X[(int64_t)r * 2 * Dr + k]); }
  __device__ cx<R> b(int k, int j) const { return Y[(int64_t)j * 2 * Dr + k]; }
  __device__ void store(int r, int j, cx<R> val) const { Ro[(int64_t)r * Dl + j] = val; }
};

template <typename R>
__global__ void k_renv_last(EnvBufs e, int n) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < e.nb) {
    cx<R> *Rl = reinterpret_cast<cx<R> *>(e.renv) + (int64_t)z * e.renv_elems + e.roff[n - 1];
    Rl[0] = mkc<R>(1, 0);
  }
}

// ---- trie level: T = L_parent X  (Dl x 2Dr),  L = (P X)^H T  (Dr x Dr)
struct LevelArgs {
  const int32_t *site, *parent, *pauli;  // level-local node arrays (device)
  int nodes;
};

template <typename R>
struct ProbL1 {
  StateView v;
  EnvBufs e;
  LevelArgs lv;
  const cx<R> *L, *X;
  cx<R> *T;
  int Dl, Dr;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M, int &N, int &K) {
    const int node = z / e.nb, zb = z - node * e.nb;
    const int par = lv.parent[node];
    if (par < 0) return false;
    const int b = e.b0 + zb, s = lv.site[node];
    Dl = dimv(v, b, s);
    Dr = dimv(v, b, s + 1);
    M = Dl;
    N = 2 * Dr;
    K = Dl;
    L = reinterpret_cast<const cx<R> *>(e.lprev) + ((int64_t)par * e.nb + zb) * e.env_elems;
    X = site_ptr<R>(v, b, s);
    T = reinterpret_cast<cx<R> *>(e.tmp) + (int64_t)z * e.tmp_elems;
    return true;
  }
  __device__ cx<R> a(int i, int k) const { return L[(int64_t)i * Dl + k]; }
  __device__ cx<R> b(int k, int j) const { return X[(int64_t)k * 2 * Dr + j]; }
  __device__ void store(int i, int j, cx<R> val) const { T[(int64_t)i * 2 * Dr + j] = val; }
};

template <typename R>
struct ProbL2 {
  StateView v;
  EnvBufs e;
  LevelArgs lv;
  unsigned long long *counters;
  const cx<R> *X, *T;
  cx<R> *Lo;
  int Dl, Dr, flip, pau;
  static constexpr bool A_KFAST = true, B_KFAST = false;
  __device__ bool setup(int z, int &M, int &N, int &K) {
    const int node = z / e.nb, zb = z - node * e.nb;
    const int b = e.b0 + zb, s = lv.site[node];
    const bool root = lv.parent[node] < 0;
    Dl = dimv(v, b, s);
    Dr = dimv(v, b, s + 1);
    M = Dr;
    N = Dr;
    K = 2 * Dl;
    pau = lv.pauli[node];
    flip = (pau == 1 || pau == 2) ? 1 : 0;
    X = site_ptr<R>(v, b, s);
    T = root ? X : reinterpret_cast<const cx<R> *>(e.tmp) + (int64_t)z * e.tmp_elems;
    Lo = reinterpret_cast<cx<R> *>(e.lcur) + ((int64_t)node * e.nb + zb) * e.env_elems;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      atomicAdd(&counters[CNT_ENV_UPDATES], 1ull);
      const unsigned long long f = 16ull * Dl * Dr * (unsigned long long)Dr +
                                   (root ? 0ull : 16ull * Dl * Dl * (unsigned long long)Dr);
      atomicAdd(&counters[CNT_ENV_FLOPS], f);
    }
    return true;
  }
  // conj((P X)[(a,s), c]) with (P X)[a,s] = ph(s) X[a, s ^ flip]
  __device__ cx<R> a(int c, int k) const {
    const int s = k & 1;
    const cx<R> x = X[(int64_t)(k ^ flip) * Dr + c];
    cx<R> y;
    if (pau == 2)       // Y: ph(0) = -i, ph(1) = +i
      y = s ? mkc<R>(-x.im, x.re) : mkc<R>(x.im, -x.re);
    else if (pau == 3)  // Z: ph(s) = (-1)^s
      y = s ? mkc<R>(-x.re, -x.im) : x;
    else
      y = x;
    return cconj(y);
  }
  __device__ cx<R> b(int k, int j) const { return T[(int64_t)k * Dr + j]; }
  __device__ void store(int i, int j, cx<R> val) const { Lo[(int64_t)i * Dr + j] = val; }
};

// <P_t> for terms attached to this level: sum_e L[e] R_b[e]
template <typename R>
__global__ void __launch_bounds__(256) k_term_dot(StateView v, EnvBufs e, const int32_t *tterm,
                                                  const int32_t *tnode, const int32_t *tsite,
                                                  int64_t n_terms, double *per_term) {
  const int t = blockIdx.x, zb = blockIdx.y;
  const int b = e.b0 + zb;
  const int node = tnode[t], site = tsite[t];
  const int D = dimv(v, b, site + 1);
  const cx<R> *L = reinterpret_cast<const cx<R> *>(e.lcur) + ((int64_t)node * e.nb + zb) * e.env_elems;
  const cx<R> *Rr = reinterpret_cast<const cx<R> *>(e.renv) + (int64_t)zb * e.renv_elems + e.roff[site];
  double acc = 0;
  for (int i = threadIdx.x; i < D * D; i += blockDim.x)
    acc += (double)L[i].re * Rr[i].re - (double)L[i].im * Rr[i].im;
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < 8; ++w) s += red[w];
    per_term[(int64_t)b * n_terms + tterm[t]] = s;
  }
}

__global__ void k_identity_terms(const int32_t *ident, int n_ident, int64_t n_terms, int batch,
                                 double *per_term) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n_ident * batch) {
    const int b = (int)(e / n_ident), t = (int)(e - (int64_t)b * n_ident);
    per_term[(int64_t)b * n_terms + ident[t]] = 1.0;
  }
}

// E[b] = sum_k c_k <P_k>, fixed term order, FP64; NaN/Inf flagged.
__global__ void k_energy(const double *per_term, const double *coeffs, int64_t n_terms, int batch,
                         double *energy, uint32_t *err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double s = 0;
  const double *pt = per_term + (int64_t)b * n_terms;
  for (int64_t k = 0; k < n_terms; ++k) s += coeffs[k] * pt[k];
  energy[b] = s;
  if (!isfinite(s)) atomicOr(err, TNMPS_EFLAG_NUMERIC);
}

struct WsLayout {
  size_t plan_bytes, per_term_off, energy_off, roff_off, renv_off, lprev_off, lcur_off, tmp_off,
      total;
  int64_t renv_elems, env_elems, tmp_elems;
  // plan sub-offsets
  size_t o_site, o_parent, o_pauli, o_tterm, o_tnode, o_tsite, o_ident, o_coeffs;
  // tensor-core form: site operand offsets/geometry, converted site operands,
  // row-K environments (lprev/lcur) and intermediates (tmp) in bytes
  bool tc;
  size_t o_tc_soff, o_tc_geo, tc_sites_off;
  int64_t tc_site_stride, tc_env_bytes;
};

static bool tc_form(const tnmps_ctx *c) { return c->dtype == TNMPS_C64_BF16SPLIT; }

// byte offset of each site's converted operands inside one state's block
static std::vector<int64_t> tc_site_offsets(const tnmps_ctx *c, int64_t *stride) {
  std::vector<int64_t> off(c->n);
  int64_t o = 0;
  for (int i = 0; i < c->n; ++i) {
    off[i] = o;
    o += swtc::site_bytes(c->cap[i], c->cap[i + 1]);
  }
  *stride = o;
  return off;
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace carving. The plan region (trie, terms, coefficients, right
// environment offsets, tensor-core site geometry) comes first and depends only
// on the context and the term set, so a cached upload stays valid for any
// chunk size. The per-term and energy result regions are reserved only when
// the caller supplies no device output for them (pt_region / e_region).
static WsLayout layout(const tnmps_ctx *c, const TermPlan &p, int bc, bool pt_region = true,
                       bool e_region = true) {
  WsLayout L{};
  const size_t esz = c->dtype == TNMPS_C128 ? 16 : 8;
  const size_t nn = p.node_site.size(), nt = p.tterm.size();
  size_t o = 0;
  L.o_site = o;
  o = al(o + 4 * nn);
  L.o_parent = o;
  o = al(o + 4 * nn);
  L.o_pauli = o;
  o = al(o + 4 * nn);
  L.o_tterm = o;
  o = al(o + 4 * nt);
  L.o_tnode = o;
  o = al(o + 4 * nt);
  L.o_tsite = o;
  o = al(o + 4 * nt);
  L.o_ident = o;
  o = al(o + 4 * p.identity_terms.size());
  L.o_coeffs = o;
  o = al(o + 8 * (size_t)p.n_terms);
  L.roff_off = o;
  o = al(o + 8 * (size_t)c->n);
  L.o_tc_soff = o;
  o = al(o + 8 * (size_t)c->n);
  L.o_tc_geo = o;
  o = al(o + 8 * (size_t)c->n);
  L.plan_bytes = o;
  L.per_term_off = o;
  if (pt_region) o = al(o + 8 * (size_t)c->batch * (size_t)p.n_terms);
  L.energy_off = o;
  if (e_region) o = al(o + 8 * (size_t)c->batch);
  int64_t re = 0;
  for (int i = 0; i < c->n; ++i) re += (int64_t)c->cap[i + 1] * c->cap[i + 1];
  L.renv_elems = re;
  L.env_elems = (int64_t)c->chi * c->chi;
  L.tmp_elems = 2 * (int64_t)c->chi * c->chi;
  L.renv_off = o;
  o = al(o + esz * (size_t)bc * (size_t)re);
  const size_t ln = p.max_level_nodes > 0 ? (size_t)p.max_level_nodes : 1;
  L.tc = tc_form(c);
  if (L.tc) {
    L.tc_env_bytes = swtc::rowk_bytes(c->chi);
    tc_site_offsets(c, &L.tc_site_stride);
    L.tc_sites_off = o;
    o = al(o + (size_t)bc * (size_t)L.tc_site_stride);
    L.lprev_off = o;
    o = al(o + ln * bc * (size_t)L.tc_env_bytes);
    L.lcur_off = o;
    o = al(o + ln * bc * (size_t)L.tc_env_bytes);
    L.tmp_off = o;
    o = al(o + ln * bc * 2 * (size_t)L.tc_env_bytes);
  } else {
    L.lprev_off = o;
    o = al(o + esz * ln * bc * (size_t)L.env_elems);
    L.lcur_off = o;
    o = al(o + esz * ln * bc * (size_t)L.env_elems);
    L.tmp_off = o;
    o = al(o + esz * ln * bc * (size_t)L.tmp_elems);
  }
  L.total = o;
  return L;
}

// The trie levels of one state chunk on the tensor cores (BF16-split form):
// convert the site tensors, seed the roots with identity environments, then
// per level the two GEMM steps and the dots of the terms ending there.
static cudaError_t run_levels_tc(tnmps_ctx *c, const TermPlan &p, const WsLayout &L, char *ws,
                                 const EnvBufs &e, const int32_t *d_site, const int32_t *d_parent,
                                 const int32_t *d_pauli, const int32_t *d_tterm,
                                 const int32_t *d_tnode, const int32_t *d_tsite, double *per_term) {
  cudaStream_t st = c->stream;
  TcSweep t{};
  t.stages = c->tuning.gemm_stages;
  t.fused = c->tuning.sweep_fused;
  t.tslots = (int64_t)((L.total - L.tmp_off) / (2 * (size_t)L.tc_env_bytes));
  t.dims = c->dims;
  t.n = c->n;
  t.b0 = e.b0;
  t.nb = e.nb;
  t.site_ops = reinterpret_cast<uint8_t *>(ws + L.tc_sites_off);
  t.site_off = reinterpret_cast<const int64_t *>(ws + L.o_tc_soff);
  t.site_geo = reinterpret_cast<const int32_t *>(ws + L.o_tc_geo);
  t.site_stride = L.tc_site_stride;
  t.lprev = reinterpret_cast<uint8_t *>(ws + L.lprev_off);
  t.lcur = reinterpret_cast<uint8_t *>(ws + L.lcur_off);
  t.tbuf = reinterpret_cast<uint8_t *>(ws + L.tmp_off);
  t.env_bytes = L.tc_env_bytes;
  t.rt = swtc::cdiv(c->chi, 128);
  t.nmax = c->chi <= 128 ? 128 : 256;
  t.err = c->err;
  cudaError_t err = tc_prep_sites(t, c->sites, c->site_off_dev, c->state_elems, st, &c->launches);
  if (err != cudaSuccess) return err;
  for (int d = 1; d <= p.depth; ++d) {
    const int64_t s0 = p.level_start[d - 1], s1 = p.level_start[d];
    const int nodes = (int)(s1 - s0);
    if (nodes == 0) continue;
    int dmax_r = 1;
    for (int64_t k = s0; k < s1; ++k) dmax_r = std::max(dmax_r, c->ub[p.node_site[k] + 1]);
    if (d == 1 && (err = tc_root_envs(t, d_site + s0, nodes, 0, st, &c->launches)) != cudaSuccess)
      return err;
    cudaEvent_t ev = prof_begin(c, PC_ENV_TC);
    if ((err = tc_level(t, d_site + s0, d_parent + s0, d_pauli + s0, nodes, d == 1, dmax_r,
                        c->counters, st, &c->launches)) != cudaSuccess)
      return err;
    prof_end(c, PC_ENV_TC, ev);
    const int64_t t0 = p.tlevel_start[d - 1], t1 = p.tlevel_start[d];
    if ((err = tc_term_dot(t, e.renv, e.roff, e.renv_elems, d_tterm + t0, d_tnode + t0,
                           d_tsite + t0, (int)(t1 - t0), p.n_terms, per_term, st,
                           &c->launches)) != cudaSuccess)
      return err;
    std::swap(t.lprev, t.lcur);
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t run_expect(tnmps_ctx *c, const TermPlan &p, char *ws, size_t ws_bytes, int chunk,
                       double *energy_dev, double *per_term_dev, double **energy_used,
                       double **per_term_used) {
  const int B = c->batch;
  int bc = chunk > 0 ? (chunk < B ? chunk : B) : B;
  const bool pt_region = per_term_dev == nullptr, e_region = energy_dev == nullptr;
  WsLayout L = layout(c, p, bc, pt_region, e_region);
  while (L.total > ws_bytes && bc > 1) {
    bc = (bc + 1) / 2;
    L = layout(c, p, bc, pt_region, e_region);
  }
  if (L.total > ws_bytes) return cudaErrorMemoryAllocation;
  cudaStream_t st = c->stream;
  cudaError_t err;
  // plan upload (skipped when the same term set was uploaded to this workspace last)
  if (c->plan_terms != (const void *)&p || c->plan_ws != (void *)ws) {
#define UP(off, vec)                                                                       \
  if (!(vec).empty()) {                                                                    \
    err = cudaMemcpyAsync(ws + (off), (vec).data(), (vec).size() * sizeof((vec)[0]),       \
                          cudaMemcpyHostToDevice, st);                                     \
    if (err != cudaSuccess) return err;                                                    \
  }
    std::vector<int32_t> pauli32(p.node_pauli.begin(), p.node_pauli.end());
    UP(L.o_site, p.node_site);
    UP(L.o_parent, p.node_parent);
    UP(L.o_pauli, pauli32);
    UP(L.o_tterm, p.tterm);
    UP(L.o_tnode, p.tnode);
    UP(L.o_tsite, p.tsite);
    UP(L.o_ident, p.identity_terms);
    UP(L.o_coeffs, p.coeffs);
    std::vector<int64_t> roff(c->n);
    int64_t o = 0;
    for (int i = 0; i < c->n; ++i) {
      roff[i] = o;
      o += (int64_t)c->cap[i + 1] * c->cap[i + 1];
    }
    UP(L.roff_off, roff);
    std::vector<int64_t> tc_soff;
    std::vector<int32_t> tc_geo;
    if (L.tc) {
      int64_t stride = 0;
      tc_soff = tc_site_offsets(c, &stride);
      tc_geo.resize(2 * (size_t)c->n);
      for (int i = 0; i < c->n; ++i) {
        tc_geo[2 * i] = swtc::cdiv(c->cap[i], swtc::KCH);
        tc_geo[2 * i + 1] = swtc::cdiv(c->cap[i + 1], 64);
      }
      UP(L.o_tc_soff, tc_soff);
      UP(L.o_tc_geo, tc_geo);
    }
#undef UP
    // pageable sources: make sure the staging finished before the vectors die
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
    c->plan_terms = &p;
    c->plan_ws = ws;
  }
  const int32_t *d_site = reinterpret_cast<const int32_t *>(ws + L.o_site);
  const int32_t *d_parent = reinterpret_cast<const int32_t *>(ws + L.o_parent);
  const int32_t *d_pauli = reinterpret_cast<const int32_t *>(ws + L.o_pauli);
  const int32_t *d_tterm = reinterpret_cast<const int32_t *>(ws + L.o_tterm);
  const int32_t *d_tnode = reinterpret_cast<const int32_t *>(ws + L.o_tnode);
  const int32_t *d_tsite = reinterpret_cast<const int32_t *>(ws + L.o_tsite);
  const int32_t *d_ident = reinterpret_cast<const int32_t *>(ws + L.o_ident);
  const double *d_coeffs = reinterpret_cast<const double *>(ws + L.o_coeffs);
  double *per_term = per_term_dev ? per_term_dev : reinterpret_cast<double *>(ws + L.per_term_off);
  double *energy = energy_dev ? energy_dev : reinterpret_cast<double *>(ws + L.energy_off);
  if (energy_used) *energy_used = energy;
  if (per_term_used) *per_term_used = per_term;

  const StateView v = c->view();
  EnvBufs e{};
  e.renv = ws + L.renv_off;
  e.roff = reinterpret_cast<const int64_t *>(ws + L.roff_off);
  e.renv_elems = L.renv_elems;
  e.lprev = ws + L.lprev_off;
  e.lcur = ws + L.lcur_off;
  e.tmp = ws + L.tmp_off;
  e.env_elems = L.env_elems;
  e.tmp_elems = L.tmp_elems;
  const int n = c->n;

  for (int b0 = 0; b0 < B; b0 += bc) {
    e.b0 = b0;
    e.nb = (B - b0) < bc ? (B - b0) : bc;
    cudaEvent_t ev = prof_begin(c, PC_ENV);
    k_renv_last<R><<<(e.nb + 255) / 256, 256, 0, st>>>(e, n);
    ++c->launches;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    for (int i = n - 2; i >= 0; --i) {
      ProbRY<R> py{};
      py.v = v;
      py.e = e;
      py.i = i;
      if ((err = launch_gemm<R>(py, 2 * c->ub[i + 1], c->ub[i + 2], e.nb, st, &c->launches)) != cudaSuccess)
        return err;
      ProbRR<R> pr{};
      pr.v = v;
      pr.e = e;
      pr.i = i;
      pr.counters = c->counters;
      if ((err = launch_gemm<R>(pr, c->ub[i + 1], c->ub[i + 1], e.nb, st, &c->launches)) != cudaSuccess)
        return err;
    }
    if (L.tc) {
      if ((err = run_levels_tc(c, p, L, ws, e, d_site, d_parent, d_pauli, d_tterm, d_tnode,
                               d_tsite, per_term)) != cudaSuccess)
        return err;
      prof_end(c, PC_ENV, ev);
      continue;
    }
    for (int d = 1; d <= p.depth; ++d) {
      const int64_t s0 = p.level_start[d - 1], s1 = p.level_start[d];
      LevelArgs lv{d_site + s0, d_parent + s0, d_pauli + s0, (int)(s1 - s0)};
      if (lv.nodes == 0) continue;
      int dmax = 1;
      for (int64_t k = s0; k < s1; ++k) {
        const int s = p.node_site[k];
        dmax = c->ub[s] > dmax ? c->ub[s] : dmax;
        dmax = c->ub[s + 1] > dmax ? c->ub[s + 1] : dmax;
      }
      if (d > 1) {
        ProbL1<R> p1{};
        p1.v = v;
        p1.e = e;
        p1.lv = lv;
        if ((err = launch_gemm<R>(p1, dmax, 2 * dmax, lv.nodes * e.nb, st, &c->launches)) != cudaSuccess)
          return err;
      }
      ProbL2<R> p2{};
      p2.v = v;
      p2.e = e;
      p2.lv = lv;
      p2.counters = c->counters;
      if ((err = launch_gemm<R>(p2, dmax, dmax, lv.nodes * e.nb, st, &c->launches)) != cudaSuccess) return err;
      const int64_t t0 = p.tlevel_start[d - 1], t1 = p.tlevel_start[d];
      if (t1 > t0) {
        dim3 grid((unsigned)(t1 - t0), e.nb);
        k_term_dot<R><<<grid, 256, 0, st>>>(v, e, d_tterm + t0, d_tnode + t0, d_tsite + t0,
                                            p.n_terms, per_term);
        ++c->launches;
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
      }
      void *tmp = e.lprev;
      e.lprev = e.lcur;
      e.lcur = tmp;
    }
    e.lprev = ws + L.lprev_off;
    e.lcur = ws + L.lcur_off;
    prof_end(c, PC_ENV, ev);
  }
  cudaEvent_t evt = prof_begin(c, PC_TERM);
  if (!p.identity_terms.empty()) {
    const int64_t cnt = (int64_t)p.identity_terms.size() * B;
    k_identity_terms<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
        d_ident, (int)p.identity_terms.size(), p.n_terms, B, per_term);
    ++c->launches;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_energy<<<(B + 127) / 128, 128, 0, st>>>(per_term, d_coeffs, p.n_terms, B, energy, c->err);
  ++c->launches;
  prof_end(c, PC_TERM, evt);
  return cudaGetLastError();
}

}  // namespace

size_t expect_ws_bytes(const tnmps_ctx *c, const TermPlan &p, int chunk, bool pt_region,
                       bool e_region) {
  const int bc = chunk > 0 ? (chunk < c->batch ? chunk : c->batch) : c->batch;
  return layout(c, p, bc, pt_region, e_region).total;
}

cudaError_t expect_run(tnmps_ctx *c, const TermPlan &p, char *ws, size_t ws_bytes, int chunk,
                       double *energy_dev, double *per_term_dev, double **energy_used,
                       double **per_term_used) {
  if (c->dtype == TNMPS_C128)
    return run_expect<double>(c, p, ws, ws_bytes, chunk, energy_dev, per_term_dev, energy_used,
                              per_term_used);
  return run_expect<float>(c, p, ws, ws_bytes, chunk, energy_dev, per_term_dev, energy_used,
                           per_term_used);
}
