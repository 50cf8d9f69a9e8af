// K5 on the fifth-generation tensor cores (dtype TNMPS_C64_BF16SPLIT): the
// transfer-matrix sweeps of the Pauli-sum expectation values (Sec. V.B
// measures every Hamiltonian term on the ansatz state; here the terms' shared
// prefixes are swept once) as BF16-split complex GEMMs with FP32 accumulation
// in tensor memory.
//
// One trie-node update, with X the site tensor (D_l, 2, D_r) and L the
// parent's left environment (D_l x D_l), is two complex products of the form
// C = A B^T (plain transpose, B stored row by row along K):
//   step 1:  T[(s,j)][i] = ph(s) sum_a X[a, s^f, j] L[i][a]
//   step 2:  L'[c][c']   = sum_{s,a} conj(X[a,s,c]) T[(s,c')][a]
// where the node's Pauli is sum_s ph(s) |s><s^f| (I, Z: f = 0; X, Y: f = 1).
// The A operands (X^T, X_s^H) are converted once per call; the B operands
// (L, T) are written by the previous step's epilogue directly in the operand
// layout, so intermediate results never leave the tile format.
//
// Real embedding of a complex product C = A B^T: with each row of B stored as
// (Re | Im) along K, the rows of the real A that produce Re C hold (Re A | -Im
// A) and those that produce Im C hold (Im A | Re A). An M tile covers 64
// complex rows: accumulator lanes 0..63 are Re C, lanes 64..127 Im C. The
// Pauli phase (+-1, +-i) only selects which K half of the destination each
// accumulator half lands in, and its sign.
//
// Split precision: every real operand value is v = hi + lo (two BF16), and
// each product is hi*hi + hi*lo + lo*hi (three MMAs; the dropped lo*lo term
// is of relative size 2^-16), accumulated in FP32.
//
// Pipeline: persistent CTAs (one per SM, 192 threads) walk the output tiles.
// One thread streams each K step's tiles (A hi/lo, B hi/lo) into a ring of
// shared-memory stages with bulk copies on the TMA unit, counted on the
// stage's mbarrier; one thread issues the stage's MMAs into one of two TMEM
// accumulators and commits them to the stage's "empty" mbarrier; four warps
// read the other accumulator with tcgen05.ld and write the split result of
// the previous tile meanwhile. Every wait is bounded: after a timeout the CTA
// flags TNMPS_EFLAG_TIMEOUT, waits (bounded) for its copies and MMAs in
// flight, frees its tensor memory and returns.
#include "sweep_tc.h"
#include "tc_util.cuh"

namespace {

using swtc::KCH;
using swtc::TILE;

__device__ __forceinline__ int dcdiv(int a, int b) { return (a + b - 1) / b; }
__device__ __forceinline__ int round32(int x) { return (x + 31) & ~31; }

__device__ __forceinline__ int dim_of(const TcSweep &t, int zb, int i) {
  return t.dims[(int64_t)(t.b0 + zb) * (t.n + 1) + i];
}

// byte offset of (row r, 16-byte K vector kv) inside a tile
__device__ __forceinline__ uint32_t tile_off(int r, int kv) {
  return (uint32_t)((r >> 3) * 1024 + kv * 128 + (r & 7) * 16);
}

// v[0..7] * sign -> the 16-byte vector (r, kv) of the hi and the lo tile
__device__ __forceinline__ void store_split8(uint8_t *hi, uint8_t *lo, int r, int kv,
                                             const float *v, float sign) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    uint16_t h0, l0, h1, l1;
    tc::bf16_split(sign * v[2 * e], h0, l0);
    tc::bf16_split(sign * v[2 * e + 1], h1, l1);
    h[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    l[e] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  }
  const uint32_t o = tile_off(r, kv);
  *reinterpret_cast<uint4 *>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4 *>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// ------------------------------------------------------------ operand prep
// Site block: A1 = X^T, tiles [chunk][piece][2 * mt_cap] (row tile s'*mt_cap +
// t covers the columns j = 64t..64t+63 of X[:, s', :]); then A2_s = X_s^H,
// tiles [s][chunk][piece][mt_cap]. Rows and K beyond the actual dimensions
// are written as zeros: the GEMMs run over whole 32-wide K chunks.
__global__ void __launch_bounds__(256) k_prep(TcSweep t, const cx<float> *sites,
                                              const int64_t *soff, int64_t state_elems) {
  const int i = blockIdx.x, zb = blockIdx.y;
  const int Dl = dim_of(t, zb, i), Dr = dim_of(t, zb, i + 1);
  const int kc_cap = t.site_geo[2 * i], mt_cap = t.site_geo[2 * i + 1];
  const int Kc = dcdiv(Dl, KCH), MT = dcdiv(Dr, 64);
  const cx<float> *X = sites + (int64_t)(t.b0 + zb) * state_elems + soff[i];
  uint8_t *base = t.site_ops + (int64_t)zb * t.site_stride + t.site_off[i];
  const int64_t a1_bytes = (int64_t)kc_cap * 2 * 2 * mt_cap * TILE;
  const int64_t items = (int64_t)4 * MT * Kc * 1024;
  for (int64_t e = threadIdx.x; e < items; e += blockDim.x) {
    const int r = (int)(e & 127);
    const int kv = (int)((e >> 7) & 7);
    int64_t rest = e >> 10;
    const int q = (int)(rest % Kc);
    rest /= Kc;
    const int tt = (int)(rest % MT);
    const int w = (int)(rest / MT);  // 0, 1: A1 for s' = w; 2, 3: A2 for s = w - 2
    const int s = w & 1;
    const int part = r >> 6;              // 0: rows of Re C, 1: rows of Im C
    const int col = tt * 64 + (r & 63);   // j (A1) or c (A2)
    const int half = kv >> 2;             // 0: Re half of K, 1: Im half
    const int a0 = q * KCH + (kv & 3) * 8;
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int a = a0 + u;
      cx<float> x = mkc<float>(0.f, 0.f);
      if (col < Dr && a < Dl) x = X[(int64_t)(a * 2 + s) * Dr + col];
      const float ar = x.re, ai = w < 2 ? x.im : -x.im;  // A1: X, A2: conj(X)
      v[u] = part == 0 ? (half == 0 ? ar : -ai) : (half == 0 ? ai : ar);
    }
    uint8_t *hi, *lo;
    if (w < 2) {
      hi = base + ((int64_t)(q * 2) * 2 * mt_cap + (s * mt_cap + tt)) * TILE;
      lo = hi + (int64_t)2 * mt_cap * TILE;
    } else {
      hi = base + a1_bytes + ((int64_t)((s * kc_cap + q) * 2) * mt_cap + tt) * TILE;
      lo = hi + (int64_t)mt_cap * TILE;
    }
    store_split8(hi, lo, r, kv, v, 1.f);
  }
}

// identity environment of size D_l(site) for each root node and state
__global__ void __launch_bounds__(256) k_root_env(TcSweep t, const int32_t *node_site) {
  const int node = blockIdx.x, zb = blockIdx.y;
  const int D = dim_of(t, zb, node_site[node]);
  uint8_t *env = t.lprev + ((int64_t)node * t.nb + zb) * t.env_bytes;
  const int rows = (D + 63) & ~63, Kc = dcdiv(D, KCH);
  const int64_t items = (int64_t)Kc * rows * 8;
  for (int64_t e = threadIdx.x; e < items; e += blockDim.x) {
    const int r = (int)(e % rows);
    const int kv = (int)((e / rows) & 7);
    const int q = (int)(e / ((int64_t)rows * 8));
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = q * KCH + (kv & 3) * 8 + u;
      v[u] = (kv < 4 && r < D && k == r) ? 1.f : 0.f;
    }
    uint8_t *hi = env + ((int64_t)(q * 2) * t.rt + r / 128) * TILE;
    store_split8(hi, hi + (int64_t)t.rt * TILE, r & 127, kv, v, 1.f);
  }
}

// ------------------------------------------------------------ the GEMM
// Addresses of one CTA's operands. K step kt = sh * kc + q reads
//   A: a + sh * a_s + q * a_kt + piece * a_pc   (one 16 KB tile)
//   B: b + sh * b_s + q * b_kt + piece * b_pc   (b_bytes = N rows x 128 B)
struct Unit {
  const uint8_t *a, *b;
  int64_t a_kt, a_pc, a_s, b_kt, b_pc, b_s;
  int kc, nk, N;
  uint32_t b_bytes;
  uint8_t *out;  // destination row-K matrix
  int row0;      // destination row of accumulator row 0 of the tile
  int half[2];   // K half of the destination for the Re / Im accumulator rows
  float sgn[2];
  unsigned long long flops;  // algorithmic flops to count for this item (0: none)
};

struct LevelArgsTc {
  const int32_t *site, *parent, *pauli;
  int nodes, grid_m;
  bool level1;
  unsigned long long *counters;
};

// step 1: T = (P X) contracted with the parent environment; M tile g covers
// s' = g / MT, columns j of tile g % MT.
struct Step1 {
  TcSweep t;
  LevelArgsTc lv;
  __device__ bool setup(int item, Unit &u) const {
    const int unit = item / lv.grid_m, g = item - unit * lv.grid_m;
    const int zb = unit / lv.nodes, node = unit - zb * lv.nodes;
    const int site = lv.site[node];
    const int Dl = dim_of(t, zb, site), Dr = dim_of(t, zb, site + 1);
    const int MT = dcdiv(Dr, 64);
    if (g >= 2 * MT) return false;
    u.flops = 0;
    const int sp = g / MT, tt = g - sp * MT;
    const int mt_cap = t.site_geo[2 * site + 1];
    const uint8_t *base = t.site_ops + (int64_t)zb * t.site_stride + t.site_off[site];
    u.a = base + (int64_t)(sp * mt_cap + tt) * TILE;
    u.a_pc = (int64_t)2 * mt_cap * TILE;
    u.a_kt = 2 * u.a_pc;
    u.a_s = 0;
    const int par = lv.level1 ? node : lv.parent[node];
    u.b = t.lprev + ((int64_t)par * t.nb + zb) * t.env_bytes;
    u.b_pc = (int64_t)t.rt * TILE;
    u.b_kt = 2 * u.b_pc;
    u.b_s = 0;
    u.kc = u.nk = dcdiv(Dl, KCH);
    u.N = round32(Dl);
    u.b_bytes = (uint32_t)u.N * 128u;
    const int pau = lv.pauli[node];
    const int f = (pau == 1 || pau == 2) ? 1 : 0;
    const int so = sp ^ f;
    // phase code of ph(so): 0: +1, 1: -1, 2: -i, 3: +i
    const int ph = pau == 3 ? (so ? 1 : 0) : pau == 2 ? (so ? 3 : 2) : 0;
    // Re rows (value ar):  +1 -> Re, +;  -1 -> Re, -;  -i -> Im, -;  +i -> Im, +
    // Im rows (value ai):  +1 -> Im, +;  -1 -> Im, -;  -i -> Re, +;  +i -> Re, -
    u.half[0] = ph >= 2 ? 1 : 0;
    u.half[1] = ph >= 2 ? 0 : 1;
    u.sgn[0] = (ph == 1 || ph == 2) ? -1.f : 1.f;
    u.sgn[1] = (ph == 1 || ph == 3) ? -1.f : 1.f;
    u.out = t.tbuf + (((int64_t)node * t.nb + zb) * 2 + so) * t.env_bytes;
    u.row0 = tt * 64;
    return true;
  }
};

// step 2: L' = sum_s X_s^H T_s; M tile g covers the rows c = 64g..64g+63.
struct Step2 {
  TcSweep t;
  LevelArgsTc lv;
  __device__ bool setup(int item, Unit &u) const {
    const int unit = item / lv.grid_m, g = item - unit * lv.grid_m;
    const int zb = unit / lv.nodes, node = unit - zb * lv.nodes;
    const int site = lv.site[node];
    const int Dl = dim_of(t, zb, site), Dr = dim_of(t, zb, site + 1);
    if (g >= dcdiv(Dr, 64)) return false;
    const int kc_cap = t.site_geo[2 * site], mt_cap = t.site_geo[2 * site + 1];
    const uint8_t *base = t.site_ops + (int64_t)zb * t.site_stride + t.site_off[site];
    const int64_t a1_bytes = (int64_t)kc_cap * 2 * 2 * mt_cap * TILE;
    u.a = base + a1_bytes + (int64_t)g * TILE;
    u.a_pc = (int64_t)mt_cap * TILE;
    u.a_kt = 2 * u.a_pc;
    u.a_s = (int64_t)kc_cap * u.a_kt;
    u.b = t.tbuf + ((int64_t)node * t.nb + zb) * 2 * t.env_bytes;
    u.b_pc = (int64_t)t.rt * TILE;
    u.b_kt = 2 * u.b_pc;
    u.b_s = t.env_bytes;
    u.kc = dcdiv(Dl, KCH);
    u.nk = 2 * u.kc;
    u.N = round32(Dr);
    u.b_bytes = (uint32_t)u.N * 128u;
    u.out = t.lcur + ((int64_t)node * t.nb + zb) * t.env_bytes;
    u.row0 = g * 64;
    u.half[0] = 0;
    u.half[1] = 1;
    u.sgn[0] = u.sgn[1] = 1.f;
    // algorithmic flops of the whole update, counted once (M tile 0); the
    // root's product with the identity is not counted
    u.flops = g == 0 ? 16ull * Dl * Dr * (unsigned long long)Dr +
                           (lv.level1 ? 0ull : 16ull * Dl * Dl * (unsigned long long)Dr)
                     : 0ull;
    return true;
  }
};

template <int NMAX>
struct Ring {
  static constexpr int S = NMAX <= 128 ? 3 : 2;
  static constexpr uint32_t A_PIECE = TILE;
  static constexpr uint32_t B_PIECE = NMAX * 128;
  static constexpr uint32_t STAGE = 2 * A_PIECE + 2 * B_PIECE;
  static constexpr int SMEM = 1024 + S * STAGE;
};

// Wait on an mbarrier phase unless another role of the CTA has failed; a
// timeout marks the CTA failed. Returns true when the phase completed.
__device__ __forceinline__ bool wait_or_fail(uint64_t *bar, uint32_t parity,
                                             volatile int *fail) {
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(bar, parity)) {
    if (*fail) return false;
    if (clock64() - t0 > 2000000000ll) {
      *fail = 1;
      return false;
    }
  }
  return true;
}

// Persistent CTAs (one per SM) walk the items (node-state, M tile)
// blockIdx.x, blockIdx.x + gridDim.x, ... with three roles:
//   warp 4 (one thread): bulk copies of every K step of every item into the
//     stage ring (a stage is refilled once the MMAs that read it completed);
//   warp 5 (one thread): the MMAs of item i into accumulator i % 2, after the
//     epilogue has drained that accumulator (item i - 2);
//   warps 0-3: the epilogue of item i (warp w reads TMEM lanes 32w..32w+31),
//     overlapping the MMAs of item i + 1.
template <class Prob, int NMAX>
__global__ void __launch_bounds__(192, 1) k_swtc(Prob p, int items, uint32_t *err) {
  using RG = Ring<NMAX>;
  constexpr int S = RG::S;
  extern __shared__ uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                            ~(uintptr_t)1023);
  __shared__ uint64_t full[S], empty[S], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t NTM = 2 * NMAX;  // two accumulators
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, NTM);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 4);
    }
    tc::mbar_init(&mma_done, 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int *fail = &s_fail;

  if (warp == 4) {
    if (lane == 0) {  // producer
      int kg = 0;     // K steps issued so far (all items)
      for (int it = blockIdx.x; it < items && !*fail; it += gridDim.x) {
        Unit u;
        if (!p.setup(it, u)) continue;
        for (int kt = 0; kt < u.nk; ++kt, ++kg) {
          const int s = kg % S;
          if (kg >= S && !wait_or_fail(&empty[s], (uint32_t)(((kg / S) - 1) & 1), fail)) break;
          const int sh = kt / u.kc, q = kt - sh * u.kc;
          const uint8_t *a = u.a + sh * u.a_s + q * u.a_kt;
          const uint8_t *b = u.b + sh * u.b_s + q * u.b_kt;
          uint8_t *st = sm + s * RG::STAGE;
          tc::mbar_arrive_expect_tx(&full[s], 2 * RG::A_PIECE + 2 * u.b_bytes);
          tc::bulk_g2s(st, a, RG::A_PIECE, &full[s]);
          tc::bulk_g2s(st + RG::A_PIECE, a + u.a_pc, RG::A_PIECE, &full[s]);
          tc::bulk_g2s(st + 2 * RG::A_PIECE, b, u.b_bytes, &full[s]);
          tc::bulk_g2s(st + 2 * RG::A_PIECE + RG::B_PIECE, b + u.b_pc, u.b_bytes, &full[s]);
        }
      }
      // every copy issued must have landed before the CTA may leave
      for (int k = kg > S ? kg - S : 0; k < kg; ++k)
        if (!tc::mbar_wait(&full[k % S], (uint32_t)((k / S) & 1))) s_fail = 1;
    }
    __syncwarp();
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int kg = 0, n = 0;  // K steps consumed, items started
      for (int it = blockIdx.x; it < items && !*fail; it += gridDim.x) {
        Unit u;
        if (!p.setup(it, u)) continue;
        const int ab = n & 1;
        if (n >= 2 && !wait_or_fail(&acc_empty[ab], (uint32_t)(((n >> 1) - 1) & 1), fail)) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(ab * NMAX);
        const uint32_t idesc = tc::idesc_bf16(128, u.N);
        bool ok = true;
        for (int kt = 0; kt < u.nk; ++kt, ++kg) {
          const int s = kg % S;
          if (!wait_or_fail(&full[s], (uint32_t)((kg / S) & 1), fail)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t a = tc::smem_u32(sm + s * RG::STAGE);
          const uint32_t al = a + RG::A_PIECE, b = a + 2 * RG::A_PIECE, bl = b + RG::B_PIECE;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint64_t ah = tc::smem_desc(a + j * 256, 128, 1024);
            const uint64_t alo = tc::smem_desc(al + j * 256, 128, 1024);
            const uint64_t bh = tc::smem_desc(b + j * 256, 128, 1024);
            const uint64_t blo = tc::smem_desc(bl + j * 256, 128, 1024);
            tc::mma_bf16(d, ah, bh, idesc, (kt > 0 || j > 0) ? 1u : 0u);
            tc::mma_bf16(d, ah, blo, idesc, 1u);
            tc::mma_bf16(d, alo, bh, idesc, 1u);
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[ab]);
        if (u.flops) {
          atomicAdd(&p.lv.counters[CNT_ENV_UPDATES], 1ull);
          atomicAdd(&p.lv.counters[CNT_ENV_FLOPS], u.flops);
        }
        ++n;
      }
      // every MMA issued must have completed before the tensor memory is freed
      tc::mma_commit(&mma_done);
      if (!tc::mbar_wait(&mma_done, 0)) s_fail = 1;
    }
    __syncwarp();
  } else {  // epilogue warps 0-3
    const int part = warp >> 1;
    int n = 0;
    for (int it = blockIdx.x; it < items && !*fail; it += gridDim.x) {
      Unit u;
      if (!p.setup(it, u)) continue;
      const int ab = n & 1;
      if (!wait_or_fail(&acc_full[ab], (uint32_t)((n >> 1) & 1), fail)) break;
      tc::fence_after_sync();
      const int row = u.row0 + (warp & 1) * 32 + lane;
      const int kvb = (part ? u.half[1] : u.half[0]) * 4;
      const float sg = part ? u.sgn[1] : u.sgn[0];
      uint8_t *rt0 = u.out + (int64_t)(row >> 7) * TILE;
      const int64_t rts = (int64_t)p.t.rt * TILE;  // next piece
      const uint32_t src = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * NMAX);
      for (int c = 0; c < u.N; c += 32) {
        float v[32];
        tc::tmem_ld32(src + (uint32_t)c, v);
        uint8_t *hi = rt0 + (int64_t)(c / KCH) * 2 * rts;
#pragma unroll
        for (int g = 0; g < 4; ++g) store_split8(hi, hi + rts, row & 127, kvb + g, v + 8 * g, sg);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                      tc::smem_u32(&acc_empty[ab]))
                                  : "memory");
      ++n;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicOr(err, TNMPS_EFLAG_TIMEOUT);
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, NTM);
}

template <class Prob, int NMAX>
cudaError_t launch_step(const Prob &p, int units, uint32_t *err, cudaStream_t s,
                        uint64_t *launches) {
  const int64_t items = (int64_t)units * p.lv.grid_m;
  if (items <= 0) return cudaSuccess;
  if (items > 0x7fffffff) return cudaErrorInvalidValue;
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm <= 0)
      n_sm = 1;
  }
  cudaError_t e = cudaFuncSetAttribute(k_swtc<Prob, NMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Ring<NMAX>::SMEM);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < n_sm ? items : n_sm);
  k_swtc<Prob, NMAX><<<grid, 192, Ring<NMAX>::SMEM, s>>>(p, (int)items, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// <P_t> = Re sum_{c,c'} L[c][c'] R[c][c'], L from the split row-K environment
__global__ void __launch_bounds__(256) k_term_dot_tc(TcSweep t, const cx<float> *renv,
                                                     const int64_t *roff, int64_t renv_elems,
                                                     const int32_t *tterm, const int32_t *tnode,
                                                     const int32_t *tsite, int64_t n_terms,
                                                     double *per_term) {
  const int k = blockIdx.x, zb = blockIdx.y;
  const int node = tnode[k], site = tsite[k];
  const int D = dim_of(t, zb, site + 1);
  const uint8_t *L = t.lcur + ((int64_t)node * t.nb + zb) * t.env_bytes;
  const cx<float> *R = renv + (int64_t)zb * renv_elems + roff[site];
  const int64_t pc = (int64_t)t.rt * TILE;
  double acc = 0;
  for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
    const int c = e / D, c2 = e - c * D;
    const int q = c2 / KCH, kk = c2 - q * KCH;
    const uint8_t *hi = L + ((int64_t)(q * 2) * t.rt + (c >> 7)) * TILE;
    const uint32_t o_re = tile_off(c & 127, kk >> 3) + (kk & 7) * 2;
    const uint32_t o_im = tile_off(c & 127, (kk + KCH) >> 3) + (kk & 7) * 2;
    auto val = [&](uint32_t o) {
      return __bfloat162float(__ushort_as_bfloat16(*reinterpret_cast<const uint16_t *>(hi + o))) +
             __bfloat162float(__ushort_as_bfloat16(*reinterpret_cast<const uint16_t *>(hi + pc + o)));
    };
    const float lr = val(o_re), li = val(o_im);
    acc += (double)lr * R[e].re - (double)li * R[e].im;
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < 8; ++w) s += red[w];
    per_term[(int64_t)(t.b0 + zb) * n_terms + tterm[k]] = s;
  }
}

}  // namespace

cudaError_t tc_prep_sites(const TcSweep &t, const void *sites, const int64_t *site_off_elems,
                          int64_t state_elems, cudaStream_t s, uint64_t *launches) {
  dim3 grid(t.n, t.nb);
  k_prep<<<grid, 256, 0, s>>>(t, reinterpret_cast<const cx<float> *>(sites), site_off_elems,
                              state_elems);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t tc_root_envs(const TcSweep &t, const int32_t *node_site, int nodes, int dmax,
                         cudaStream_t s, uint64_t *launches) {
  (void)dmax;
  if (nodes <= 0) return cudaSuccess;
  k_root_env<<<dim3(nodes, t.nb), 256, 0, s>>>(t, node_site);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t tc_level(const TcSweep &t, const int32_t *node_site, const int32_t *node_parent,
                     const int32_t *node_pauli, int nodes, bool level1, int dmax_r,
                     unsigned long long *counters, cudaStream_t s, uint64_t *launches) {
  if (nodes <= 0) return cudaSuccess;
  const int mt = swtc::cdiv(dmax_r, 64);
  LevelArgsTc lv{node_site, node_parent, node_pauli, nodes, 2 * mt, level1, counters};
  const int units = nodes * t.nb;
  cudaError_t e;
  Step1 p1{t, lv};
  e = t.nmax <= 128 ? launch_step<Step1, 128>(p1, units, t.err, s, launches)
                    : launch_step<Step1, 256>(p1, units, t.err, s, launches);
  if (e != cudaSuccess) return e;
  lv.grid_m = mt;
  Step2 p2{t, lv};
  return t.nmax <= 128 ? launch_step<Step2, 128>(p2, units, t.err, s, launches)
                       : launch_step<Step2, 256>(p2, units, t.err, s, launches);
}

cudaError_t tc_term_dot(const TcSweep &t, const void *renv, const int64_t *roff,
                        int64_t renv_elems, const int32_t *tterm, const int32_t *tnode,
                        const int32_t *tsite, int count, int64_t n_terms, double *per_term,
                        cudaStream_t s, uint64_t *launches) {
  if (count <= 0) return cudaSuccess;
  k_term_dot_tc<<<dim3(count, t.nb), 256, 0, s>>>(t, reinterpret_cast<const cx<float> *>(renv),
                                                  roff, renv_elems, tterm, tnode, tsite,
                                                  n_terms, per_term);
  if (launches) ++*launches;
  return cudaGetLastError();
}
