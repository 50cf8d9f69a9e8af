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
// The GEMM machinery (operand formats, real embedding, split products, the
// persistent warp-specialised tcgen05 pipeline) is cgemm_tc.cuh; this file
// holds the sweep's operand conversion, its two GEMM problems with their
// epilogues, and the term dots. The Pauli phase (+-1, +-i) only selects which
// K half of the destination each accumulator half lands in, and its sign.
#include "cgemm_tc.cuh"

namespace {

using ctc::dcdiv;
using ctc::round32;
using ctc::store_split8;
using ctc::tile_off;
using ctc::Unit;
using swtc::KCH;
using swtc::TILE;

__device__ __forceinline__ int dim_of(const TcSweep &t, int zb, int i) {
  return t.dims[(int64_t)(t.b0 + zb) * (t.n + 1) + i];
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

// ------------------------------------------------------------ the GEMM problems
struct LevelArgsTc {
  const int32_t *site, *parent, *pauli;
  int nodes, grid_m;
  bool level1;
  unsigned long long *counters;
};

// Epilogue shared by both steps: the accumulator row of this thread (Re or
// Im part of one complex row) goes to its K half of the destination row-K
// matrix as split BF16, 32 columns = one K chunk at a time.
__device__ __forceinline__ void rowk_epi(const Unit &u, int warp, int lane, int c,
                                         const float (&v)[32], int rt) {
  const int part = warp >> 1;
  const int row = u.row0 + (warp & 1) * 32 + lane;
  const int kvb = (part ? u.half[1] : u.half[0]) * 4;
  const float sg = part ? u.sgn[1] : u.sgn[0];
  const int64_t rts = (int64_t)rt * TILE;  // next piece
  uint8_t *hi = u.out + (int64_t)(row >> 7) * TILE + (int64_t)(c / KCH) * 2 * rts;
#pragma unroll
  for (int g = 0; g < 4; ++g) store_split8(hi, hi + rts, row & 127, kvb + g, v + 8 * g, sg);
}

__device__ __forceinline__ void count_update(const Unit &u, unsigned long long *counters) {
  if (u.flops) {
    atomicAdd(&counters[CNT_ENV_UPDATES], 1ull);
    atomicAdd(&counters[CNT_ENV_FLOPS], u.flops);
  }
}

// step 1: T = (P X) contracted with the parent environment; M tile g covers
// s' = g / MT, columns j of tile g % MT.
struct Step1 {
  TcSweep t;
  LevelArgsTc lv;
  static constexpr int PIECES = 2, EPI_SMEM = 0;
  __device__ void epi(const Unit &u, int warp, int lane, int c, const float (&v)[32],
                      uint8_t *) const {
    rowk_epi(u, warp, lane, c, v, t.rt);
  }
  __device__ void done(const Unit &u) const { count_update(u, lv.counters); }
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
  static constexpr int PIECES = 2, EPI_SMEM = 0;
  __device__ void epi(const Unit &u, int warp, int lane, int c, const float (&v)[32],
                      uint8_t *) const {
    rowk_epi(u, warp, lane, c, v, t.rt);
  }
  __device__ void done(const Unit &u) const { count_update(u, lv.counters); }
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

// ------------------------------------------------------------ fused level
// Both steps of a trie level in one persistent launch. CTA c takes the
// (state, node) units c, c + G, c + 2G, ... (G CTAs) and runs, for its k-th
// unit, the step-1 M tiles of unit k and then the step-2 M tiles of unit
// k - 1: step 2 of a unit starts one unit later, while step 1 of the next
// unit keeps the tensor pipe busy. The unit's intermediate T goes to one of
// two T slots of the CTA (slot k & 1) instead of a per-unit buffer, so it is
// written and read back by the same SM within about one unit's time and
// stays in L2. The hand-off: the epilogue warps store T (generic proxy),
// fence it for the async proxy and arrive on the slot's mbarrier; the
// producer waits on it before its bulk copies read T. A slot is rewritten
// two units later, after the MMAs that read it have completed (their
// completion precedes the accumulator that the rewriting epilogue waits for).
// Roles and bounded waits as in ctc::k_cgemm.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

struct FusedItem {
  int unit, step, g, k;  // step 1 or 2; k: index of the unit in this CTA's sequence
};

// calls f(item) for this CTA's item sequence in order; f returns false to stop
template <class F>
__device__ __forceinline__ void for_items(int units, int grid_m1, int grid_m2, F f) {
  const int G = gridDim.x, c = blockIdx.x;
  const int K = c < units ? (units - c + G - 1) / G : 0;
  for (int k = 0; k <= K; ++k) {
    if (k < K)
      for (int g = 0; g < grid_m1; ++g)
        if (!f(FusedItem{c + k * G, 1, g, k})) return;
    if (k >= 1)
      for (int g = 0; g < grid_m2; ++g)
        if (!f(FusedItem{c + (k - 1) * G, 2, g, k - 1})) return;
  }
}

template <int NMAX>
__global__ void __launch_bounds__(192, 1) k_sweep_fused(Step1 p1, Step2 p2, int units,
                                                        uint32_t *err) {
  constexpr int P = 2;
  using RG = ctc::Ring<NMAX, 0, P, 3>;
  constexpr int S = RG::S;
  extern __shared__ uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                            ~(uintptr_t)1023);
  __shared__ uint64_t full[S], empty[S], acc_full[2], acc_empty[2], mma_done, t_ready[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t NTM = 2 * NMAX;
  const int gm1 = p1.lv.grid_m, gm2 = p2.lv.grid_m;
  const TcSweep &t = p1.t;
  auto setup = [&](const FusedItem &it, Unit &u) {
    bool ok;
    if (it.step == 1) {
      ok = p1.setup(it.unit * gm1 + it.g, u);
      if (ok)  // T half s' of the slot (setup put it in the per-unit buffer)
        u.out = t.tbuf + ((int64_t)(blockIdx.x * 2 + (it.k & 1)) * 2 +
                          (u.out - t.tbuf) / t.env_bytes % 2) * t.env_bytes;
    } else {
      ok = p2.setup(it.unit * gm2 + it.g, u);
      if (ok) u.b = t.tbuf + (int64_t)(blockIdx.x * 2 + (it.k & 1)) * 2 * t.env_bytes;
    }
    return ok;
  };
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, NTM);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int q = 0; q < S; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], 4);
      tc::mbar_init(&t_ready[b], 4);
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
      int kg = 0;
      int waited = -1;  // last unit index whose T hand-off was awaited
      for_items(units, gm1, gm2, [&](const FusedItem &it) {
        if (*fail) return false;
        Unit u;
        if (!setup(it, u)) return true;
        if (it.step == 2 && it.k != waited) {
          if (!ctc::wait_or_fail(&t_ready[it.k & 1], (uint32_t)((it.k >> 1) & 1), fail))
            return false;
          waited = it.k;
        }
        for (int kt = 0; kt < u.nk; ++kt, ++kg) {
          const int q = kg % S;
          if (kg >= S && !ctc::wait_or_fail(&empty[q], (uint32_t)(((kg / S) - 1) & 1), fail))
            return false;
          const int sh = kt / u.kc, qq = kt - sh * u.kc;
          const uint8_t *a = u.a + sh * u.a_s + qq * u.a_kt;
          const uint8_t *b = u.b + sh * u.b_s + qq * u.b_kt;
          uint8_t *st = sm + q * RG::STAGE;
          tc::mbar_arrive_expect_tx(&full[q], P * (RG::A_PIECE + u.b_bytes));
#pragma unroll
          for (int pc = 0; pc < P; ++pc) {
            tc::bulk_g2s(st + pc * RG::A_PIECE, a + pc * u.a_pc, RG::A_PIECE, &full[q]);
            tc::bulk_g2s(st + P * RG::A_PIECE + pc * RG::B_PIECE, b + pc * u.b_pc, u.b_bytes,
                         &full[q]);
          }
        }
        return true;
      });
      for (int k = kg > S ? kg - S : 0; k < kg; ++k)
        if (!tc::mbar_wait(&full[k % S], (uint32_t)((k / S) & 1))) s_fail = 1;
    }
    __syncwarp();
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int kg = 0, n = 0;
      for_items(units, gm1, gm2, [&](const FusedItem &it) {
        if (*fail) return false;
        Unit u;
        if (!setup(it, u)) return true;
        const int ab = n & 1;
        if (n >= 2 && !ctc::wait_or_fail(&acc_empty[ab], (uint32_t)(((n >> 1) - 1) & 1), fail))
          return false;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(ab * NMAX);
        const uint32_t idesc = tc::idesc_bf16(128, u.N);
        for (int kt = 0; kt < u.nk; ++kt, ++kg) {
          const int q = kg % S;
          if (!ctc::wait_or_fail(&full[q], (uint32_t)((kg / S) & 1), fail)) return false;
          tc::fence_after_sync();
          const uint32_t a = tc::smem_u32(sm + q * RG::STAGE);
          const uint32_t b = a + P * RG::A_PIECE;
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int o = 0; o < P; ++o)
#pragma unroll
              for (int pa = 0; pa <= o; ++pa) {
                const uint64_t ad = tc::smem_desc(a + pa * RG::A_PIECE + j * 256, 128, 1024);
                const uint64_t bd =
                    tc::smem_desc(b + (o - pa) * RG::B_PIECE + j * 256, 128, 1024);
                tc::mma_bf16(d, ad, bd, idesc, (kt > 0 || j > 0 || o > 0) ? 1u : 0u);
              }
          tc::mma_commit(&empty[q]);
        }
        tc::mma_commit(&acc_full[ab]);
        if (it.step == 2) p2.done(u);
        ++n;
        return true;
      });
      tc::mma_commit(&mma_done);
      if (!tc::mbar_wait(&mma_done, 0)) s_fail = 1;
    }
    __syncwarp();
  } else {  // epilogue warps 0-3
    int n = 0;
    for_items(units, gm1, gm2, [&](const FusedItem &it) {
      if (*fail) return false;
      Unit u;
      if (setup(it, u)) {
        const int ab = n & 1;
        if (!ctc::wait_or_fail(&acc_full[ab], (uint32_t)((n >> 1) & 1), fail)) return false;
        tc::fence_after_sync();
        const uint32_t src = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * NMAX);
        for (int c = 0; c < u.N; c += 32) {
          float v[32];
          tc::tmem_ld32(src + (uint32_t)c, v);
          rowk_epi(u, warp, lane, c, v, t.rt);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                           tc::smem_u32(&acc_empty[ab]))
                       : "memory");
        ++n;
      }
      // after the unit's last step-1 tile: hand T over to the producer
      if (it.step == 1 && it.g == gm1 - 1) {
        fence_proxy_async_global();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                           tc::smem_u32(&t_ready[it.k & 1]))
                       : "memory");
      }
      return true;
    });
  }
  tc::fence_before_sync();
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicOr(err, TNMPS_EFLAG_TIMEOUT);
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, NTM);
}

template <int NMAX>
cudaError_t launch_fused(const Step1 &p1, const Step2 &p2, int units, uint32_t *err,
                         cudaStream_t s, uint64_t *launches) {
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm <= 0)
      n_sm = 1;
  }
  constexpr int SMEM = ctc::Ring<NMAX, 0, 2, 3>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_sweep_fused<NMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  // two T slots per CTA, each of two halves, inside the workspace's T region
  int grid = n_sm < units ? n_sm : units;
  const int64_t slot_cap = p1.t.tslots / 2;
  if (grid > slot_cap) grid = (int)slot_cap;
  if (grid < 1) return cudaErrorInvalidValue;
  k_sweep_fused<NMAX><<<grid, 192, SMEM, s>>>(p1, p2, units, err);
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
  if (t.fused) {  // both steps in one launch, T kept in per-CTA slots
    LevelArgsTc lv2 = lv;
    lv2.grid_m = mt;
    Step2 p2{t, lv2};
    return t.nmax <= 128 ? launch_fused<128>(p1, p2, units, t.err, s, launches)
                         : launch_fused<256>(p1, p2, units, t.err, s, launches);
  }
  e = t.nmax <= 128
          ? ctc::launch_cgemm<Step1, 128>(p1, (int64_t)units * lv.grid_m, t.err, s, launches,
                                          t.stages)
          : ctc::launch_cgemm<Step1, 256>(p1, (int64_t)units * lv.grid_m, t.err, s, launches,
                                          t.stages);
  if (e != cudaSuccess) return e;
  lv.grid_m = mt;
  Step2 p2{t, lv};
  return t.nmax <= 128
             ? ctc::launch_cgemm<Step2, 128>(p2, (int64_t)units * lv.grid_m, t.err, s, launches,
                                             t.stages)
             : ctc::launch_cgemm<Step2, 256>(p2, (int64_t)units * lv.grid_m, t.err, s, launches,
                                             t.stages);
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
