// K2 on the fifth-generation tensor cores (dtype TNMPS_C64_BF16SPLIT): the
// two-site block of a two-qubit gate (Sec. II, Fig. "mpssvd"; Sec. IV: the
// gate acts on the pair of site tensors contracted over their shared bond),
//     Theta[(a,s1)][(s2,b)] = sum_m C_l[a,s1,m] B_{l+1}[m,s2,b],
// as a split-precision complex GEMM C = A B^T (cgemm_tc.cuh) with
//     A = C_l as rows (a,s1) along K = m   (real-embedded, converted per gate)
//     B = rows (s2,b) along K = m          (row-K, converted per gate)
// and an FP32 row-major result in theta_buf, where the fused 4x4 gate and the
// Jacobi copy are then applied (k_apply_gate4) exactly as in the FP32 form.
//
// Three BF16 pieces per value (the whole FP32 mantissa, six piece products):
// the block feeds the state itself, so its rounding compounds over every
// gate of the circuit; with two pieces (2^-16 per product) the 8-qubit
// workload's energies missed the 1e-6 sum|c_k| target (1.8e-6).
//
// The epilogue stages each 64 x 32 complex block through shared memory so
// that consecutive threads store consecutive complex elements of a row.
#include "cgemm_tc.cuh"

namespace {

using ctc::dcdiv;
using ctc::round32;
using ctc::store_pieces8;
using ctc::Unit;

constexpr int PC = 3;  // BF16 pieces per operand value
using swtc::KCH;
using swtc::TILE;

// capacity geometry: rows of A <= 2 chi (tiles of 64 complex rows), rows of
// B <= 2 chi (tiles of 128), K <= chi (chunks of 32)
__host__ __device__ inline int a_tiles(int chi) { return (2 * chi + 63) / 64; }
__host__ __device__ inline int b_tiles(int chi) { return (2 * chi + 127) / 128; }
__host__ __device__ inline int k_chunks(int chi) { return (chi + 31) / 32; }

struct ThetaArgs {
  const cx<float> *sites;
  const int64_t *site_off;
  const int32_t *dims;
  int64_t state_elems;
  int n, l, chi;
  uint8_t *A, *B;
  int64_t a_stride, b_stride;
  float *theta;  // theta_buf as interleaved complex64
  int64_t tw;
  const cx<float> *theta_in;  // theta_buf as the split's B operand source
};

__device__ __forceinline__ int dimb(const ThetaArgs &t, int b, int i) {
  return t.dims[(int64_t)b * (t.n + 1) + i];
}

// Convert C_l and B_{l+1} of state blockIdx.y into the A and B tiles; rows
// and K beyond the actual dimensions (up to whole tiles / chunks) are zeros.
__global__ void __launch_bounds__(256) k_theta_prep(ThetaArgs t) {
  const int b = blockIdx.y;
  const int Dl = dimb(t, b, t.l), Dm = dimb(t, b, t.l + 1), Dr = dimb(t, b, t.l + 2);
  const int MT = dcdiv(2 * Dl, 64), Kc = dcdiv(Dm, KCH);
  const int RT = dcdiv(round32(2 * Dr), 128);
  const int mtc = a_tiles(t.chi), rtc = b_tiles(t.chi);
  const cx<float> *C = t.sites + (int64_t)b * t.state_elems + t.site_off[t.l];
  const cx<float> *Bs = t.sites + (int64_t)b * t.state_elems + t.site_off[t.l + 1];
  uint8_t *A = t.A + (int64_t)b * t.a_stride;
  uint8_t *B = t.B + (int64_t)b * t.b_stride;
  const int64_t na = (int64_t)MT * Kc * 1024, nbv = (int64_t)RT * Kc * 1024;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nbv;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool isA = e < na;
    const int64_t f = isA ? e : e - na;
    const int r = (int)(f & 127), kv = (int)((f >> 7) & 7);
    const int64_t rest = f >> 10;
    const int q = (int)(rest % Kc), tile = (int)(rest / Kc);
    const int half = kv >> 2;
    const int m0 = q * KCH + (kv & 3) * 8;
    float v[8];
    if (isA) {
      const int part = r >> 6, i = tile * 64 + (r & 63);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int m = m0 + u;
        const cx<float> x = (i < 2 * Dl && m < Dm) ? C[(int64_t)i * Dm + m] : mkc<float>(0.f, 0.f);
        v[u] = part == 0 ? (half == 0 ? x.re : -x.im) : (half == 0 ? x.im : x.re);
      }
      store_pieces8<PC>(A + ((int64_t)(q * PC) * mtc + tile) * TILE, (int64_t)mtc * TILE, r, kv, v,
                        1.f);
    } else {
      const int j = tile * 128 + r;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int m = m0 + u;
        const cx<float> x =
            (j < 2 * Dr && m < Dm) ? Bs[(int64_t)m * 2 * Dr + j] : mkc<float>(0.f, 0.f);
        v[u] = half == 0 ? x.re : x.im;
      }
      store_pieces8<PC>(B + ((int64_t)(q * PC) * rtc + tile) * TILE, (int64_t)rtc * TILE, r, kv, v,
                        1.f);
    }
  }
}

template <int NMAX>
struct ThetaProb {
  ThetaArgs t;
  int grid_m, grid_n;  // M and N tiles per state (upper bounds)
  static constexpr int PIECES = PC, EPI_SMEM = 4 * 32 * 33 * 4;
  __device__ bool setup(int item, Unit &u) const {
    const int per = grid_m * grid_n;
    const int b = item / per, rest = item - b * per;
    const int g = rest / grid_n, nt = rest - g * grid_n;
    const int Dl = dimb(t, b, t.l), Dm = dimb(t, b, t.l + 1), Dr = dimb(t, b, t.l + 2);
    if (g >= dcdiv(2 * Dl, 64)) return false;
    const int npad = round32(2 * Dr);
    if (nt * NMAX >= npad) return false;
    const int mtc = a_tiles(t.chi), rtc = b_tiles(t.chi);
    u.a = t.A + (int64_t)b * t.a_stride + (int64_t)g * TILE;
    u.a_pc = (int64_t)mtc * TILE;
    u.a_kt = PC * u.a_pc;
    u.a_s = 0;
    u.b = t.B + (int64_t)b * t.b_stride + (int64_t)(nt * (NMAX / 128)) * TILE;
    u.b_pc = (int64_t)rtc * TILE;
    u.b_kt = PC * u.b_pc;
    u.b_s = 0;
    u.kc = u.nk = dcdiv(Dm, KCH);
    u.N = min(NMAX, npad - nt * NMAX);
    u.b_bytes = (uint32_t)u.N * 128u;
    u.out = reinterpret_cast<uint8_t *>(t.theta + 2 * (int64_t)b * t.tw);
    u.row0 = g * 64;
    u.col0 = nt * NMAX;
    u.rows = 2 * Dl;
    u.cols = 2 * Dr;
    u.flops = 0;
    return true;
  }
  // Re rows of the block are accumulator lanes 0..63 (warps 0, 1), Im rows
  // lanes 64..127 (warps 2, 3): stage the 128 x 32 slab, then write complex
  // pairs row by row.
  __device__ void epi(const Unit &u, int warp, int lane, int c, const float (&v)[32],
                      uint8_t *stage) const {
    float *T = reinterpret_cast<float *>(stage);
    const int tl = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) T[tl * 33 + j] = v[j];
    asm volatile("bar.sync 1, 128;" ::: "memory");
    cx<float> *out = reinterpret_cast<cx<float> *>(u.out);
#pragma unroll 4
    for (int e = 0; e < 16; ++e) {
      const int idx = e * 128 + tl;
      const int rr = idx >> 5, j = idx & 31;
      const int i = u.row0 + rr, col = u.col0 + c + j;
      if (i < u.rows && col < u.cols)
        out[(int64_t)i * u.cols + col] = mkc<float>(T[rr * 33 + j], T[(64 + rr) * 33 + j]);
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
  }
  __device__ void done(const Unit &) const {}
};

// ---------------------------------------------------------------- K4 split
// C_{l+1} = U_k^H Theta (k x 2Dr), the right factor of the split, as the same
// split-precision C = A B^T with
//     A = U_k^H as rows kappa < k along K = (a,s1) < 2Dl (U_k: site l, ld k)
//     B = rows (s2,c) < 2Dr along K = (a,s1)           (Theta: theta_buf)
// and the FP32 result written into site l+1 (ld 2Dr). Three pieces, as K2:
// C_{l+1} is the next centre of the state.
__host__ __device__ inline int sa_tiles(int chi) { return (chi + 63) / 64; }
__host__ __device__ inline int sk_chunks(int chi) { return (2 * chi + 31) / 32; }

__global__ void __launch_bounds__(256) k_split_prep(ThetaArgs t) {
  const int b = blockIdx.y;
  const int Dl = dimb(t, b, t.l), k = dimb(t, b, t.l + 1), Dr = dimb(t, b, t.l + 2);
  const int M2 = 2 * Dl, N2 = 2 * Dr;
  const int MT = dcdiv(k, 64), Kc = dcdiv(M2, KCH);
  const int RT = dcdiv(round32(N2), 128);
  const int mtc = sa_tiles(t.chi), rtc = b_tiles(t.chi);
  const cx<float> *U = t.sites + (int64_t)b * t.state_elems + t.site_off[t.l];
  const cx<float> *Th = t.theta_in + (int64_t)b * t.tw;
  uint8_t *A = t.A + (int64_t)b * t.a_stride;
  uint8_t *B = t.B + (int64_t)b * t.b_stride;
  const int64_t na = (int64_t)MT * Kc * 1024, nbv = (int64_t)RT * Kc * 1024;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nbv;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool isA = e < na;
    const int64_t f = isA ? e : e - na;
    const int r = (int)(f & 127), kv = (int)((f >> 7) & 7);
    const int64_t rest = f >> 10;
    const int q = (int)(rest % Kc), tile = (int)(rest / Kc);
    const int half = kv >> 2;
    const int m0 = q * KCH + (kv & 3) * 8;
    float v[8];
    if (isA) {  // conj(U[i][kappa]) along K = i
      const int part = r >> 6, kap = tile * 64 + (r & 63);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = m0 + u;
        cx<float> x = (kap < k && i < M2) ? U[(int64_t)i * k + kap] : mkc<float>(0.f, 0.f);
        x.im = -x.im;
        v[u] = part == 0 ? (half == 0 ? x.re : -x.im) : (half == 0 ? x.im : x.re);
      }
      store_pieces8<PC>(A + ((int64_t)(q * PC) * mtc + tile) * TILE, (int64_t)mtc * TILE, r, kv, v,
                        1.f);
    } else {  // Theta[i][j] along K = i
      const int j = tile * 128 + r;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = m0 + u;
        const cx<float> x = (j < N2 && i < M2) ? Th[(int64_t)i * N2 + j] : mkc<float>(0.f, 0.f);
        v[u] = half == 0 ? x.re : x.im;
      }
      store_pieces8<PC>(B + ((int64_t)(q * PC) * rtc + tile) * TILE, (int64_t)rtc * TILE, r, kv, v,
                        1.f);
    }
  }
}

template <int NMAX>
struct SplitProb : ThetaProb<NMAX> {
  __device__ bool setup(int item, Unit &u) const {
    const ThetaArgs &t = this->t;
    const int per = this->grid_m * this->grid_n;
    const int b = item / per, rest = item - b * per;
    const int g = rest / this->grid_n, nt = rest - g * this->grid_n;
    const int Dl = dimb(t, b, t.l), k = dimb(t, b, t.l + 1), Dr = dimb(t, b, t.l + 2);
    if (g >= dcdiv(k, 64)) return false;
    const int npad = round32(2 * Dr);
    if (nt * NMAX >= npad) return false;
    const int mtc = sa_tiles(t.chi), rtc = b_tiles(t.chi);
    u.a = t.A + (int64_t)b * t.a_stride + (int64_t)g * TILE;
    u.a_pc = (int64_t)mtc * TILE;
    u.a_kt = PC * u.a_pc;
    u.a_s = 0;
    u.b = t.B + (int64_t)b * t.b_stride + (int64_t)(nt * (NMAX / 128)) * TILE;
    u.b_pc = (int64_t)rtc * TILE;
    u.b_kt = PC * u.b_pc;
    u.b_s = 0;
    u.kc = u.nk = dcdiv(2 * Dl, KCH);
    u.N = min(NMAX, npad - nt * NMAX);
    u.b_bytes = (uint32_t)u.N * 128u;
    u.out = reinterpret_cast<uint8_t *>(
        const_cast<cx<float> *>(t.sites + (int64_t)b * t.state_elems + t.site_off[t.l + 1]));
    u.row0 = g * 64;
    u.col0 = nt * NMAX;
    u.rows = k;
    u.cols = 2 * Dr;
    u.flops = 0;
    return true;
  }
};

}  // namespace

// operand bytes per state: the larger of K2 (A: 2chi rows, K = chi) and the
// split (A: chi rows, K = 2chi; B: K = 2chi)
int64_t theta_tc_a_bytes(int chi) {
  const int64_t k2 = (int64_t)k_chunks(chi) * PC * a_tiles(chi) * TILE;
  const int64_t sp = (int64_t)sk_chunks(chi) * PC * sa_tiles(chi) * TILE;
  return k2 > sp ? k2 : sp;
}
int64_t theta_tc_b_bytes(int chi) {
  const int64_t k2 = (int64_t)k_chunks(chi) * PC * b_tiles(chi) * TILE;
  const int64_t sp = (int64_t)sk_chunks(chi) * PC * b_tiles(chi) * TILE;
  return k2 > sp ? k2 : sp;
}

cudaError_t launch_split_tc(tnmps_ctx *c, int l, int kub) {
  ThetaArgs t{};
  t.sites = reinterpret_cast<const cx<float> *>(c->sites);
  t.site_off = c->site_off_dev;
  t.dims = c->dims;
  t.state_elems = c->state_elems;
  t.n = c->n;
  t.l = l;
  t.chi = c->chi;
  t.A = reinterpret_cast<uint8_t *>(c->tc_a);
  t.B = reinterpret_cast<uint8_t *>(c->tc_b);
  t.a_stride = c->tc_a_stride;
  t.b_stride = c->tc_b_stride;
  t.theta_in = reinterpret_cast<const cx<float> *>(c->theta_buf);
  t.tw = c->tw;
  k_split_prep<<<dim3(8, c->batch), 256, 0, c->stream>>>(t);
  ++c->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int gm = (kub + 63) / 64;
  const int npad = (2 * c->ub[l + 2] + 31) & ~31;
  const int gn = (npad + 127) / 128;
  SplitProb<128> p{};
  p.t = t;
  p.grid_m = gm;
  p.grid_n = gn;
  return ctc::launch_cgemm<SplitProb<128>, 128>(p, (int64_t)c->batch * gm * gn, c->err, c->stream,
                                                &c->launches, c->tuning.gemm_stages);
}

cudaError_t launch_theta_tc(tnmps_ctx *c, int l) {
  ThetaArgs t{};
  t.sites = reinterpret_cast<const cx<float> *>(c->sites);
  t.site_off = c->site_off_dev;
  t.dims = c->dims;
  t.state_elems = c->state_elems;
  t.n = c->n;
  t.l = l;
  t.chi = c->chi;
  t.A = reinterpret_cast<uint8_t *>(c->tc_a);
  t.B = reinterpret_cast<uint8_t *>(c->tc_b);
  t.a_stride = c->tc_a_stride;
  t.b_stride = c->tc_b_stride;
  t.theta = reinterpret_cast<float *>(c->theta_buf);
  t.tw = c->tw;
  k_theta_prep<<<dim3(8, c->batch), 256, 0, c->stream>>>(t);
  ++c->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int gm = (2 * c->ub[l] + 63) / 64;
  const int npad = (2 * c->ub[l + 2] + 31) & ~31;
  const int gn = (npad + 127) / 128;  // 128-wide N tiles: three pieces fill the stages
  ThetaProb<128> p{t, gm, gn};
  return ctc::launch_cgemm<ThetaProb<128>, 128>(p, (int64_t)c->batch * gm * gn, c->err, c->stream,
                                                &c->launches, c->tuning.gemm_stages);
}
