// Split-precision complex GEMM  C = A B^T  (plain transpose) on the
// fifth-generation tensor cores, shared by the two-site block contraction
// (K2) and the transfer-matrix sweeps (K5) of the BF16-split form.
//
// Operand formats (16 KB tiles of 128 rows x 64 BF16 of K in the canonical
// no-swizzle K-major core-matrix order, hi and lo pieces):
//   A, real-embedded: 64 complex rows per tile; tile rows 0..63 produce Re C
//     and hold (Re A | -Im A) along each 64-wide K chunk, rows 64..127 produce
//     Im C and hold (Im A | Re A);
//   B, row-K: each row holds (Re B | Im B) per chunk of 32 complex K values.
// Accumulator lanes 0..63 of an M tile are then Re C, lanes 64..127 Im C.
//
// Split precision: every real operand value is a sum of P BF16 pieces
// (P = 2: hi + lo, 2^-18 relative; P = 3: hi + mid + lo, the whole FP32
// mantissa), and each product keeps the piece products of total order < P:
// three MMAs for P = 2 (the dropped lo*lo term is of relative size 2^-16), six
// for P = 3 (dropped terms below 2^-24), accumulated in FP32 in tensor memory.
//
// Pipeline: persistent CTAs (one per SM, 192 threads) walk the output tiles
// ("items") of the problem. One thread streams each K step's tiles (A hi/lo,
// B hi/lo) into a ring of shared-memory stages with bulk copies on the TMA
// unit, counted on the stage's mbarrier; one thread issues the stage's MMAs
// into one of two TMEM accumulators and commits them to the stage's "empty"
// mbarrier; four warps read the other accumulator with tcgen05.ld and hand
// it to the problem's epilogue, overlapping the next tile's MMAs. Every wait
// is bounded: after a timeout the CTA flags TNMPS_EFLAG_TIMEOUT, waits
// (bounded) for its copies and MMAs in flight, frees its tensor memory and
// returns.
//
// A problem provides
//   static constexpr int PIECES;                 BF16 pieces per operand value
//   static constexpr int EPI_SMEM;               bytes of epilogue staging
//   bool setup(int item, Unit &u) const;         false: nothing to do
//   void epi(const Unit &u, int warp, int lane, int col, const float (&v)[32],
//            uint8_t *stage) const;              columns col..col+31 of the
//                                                accumulator lane of this thread
//   void done(const Unit &u) const;              once per item (MMA thread)
#pragma once
#include "sweep_tc.h"
#include "tc_util.cuh"

namespace ctc {

using swtc::KCH;
using swtc::TILE;

__device__ __forceinline__ int dcdiv(int a, int b) { return (a + b - 1) / b; }
__device__ __forceinline__ int round32(int x) { return (x + 31) & ~31; }

// byte offset of (row r, 16-byte K vector kv) inside a tile
__device__ __forceinline__ uint32_t tile_off(int r, int kv) {
  return (uint32_t)((r >> 3) * 1024 + kv * 128 + (r & 7) * 16);
}

// v[0..7] * sign -> the 16-byte vector (r, kv) of the P piece tiles, piece p
// at t0 + p * pstride: v = piece_0 + piece_1 + ..., each piece the BF16 (RN)
// of what the earlier pieces left
template <int P>
__device__ __forceinline__ void store_pieces8(uint8_t *t0, int64_t pstride, int r, int kv,
                                              const float *v, float sign) {
  float rem[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) rem[e] = sign * v[e];
  const uint32_t o = tile_off(r, kv);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 b0 = __float2bfloat16_rn(rem[2 * e]);
      const __nv_bfloat16 b1 = __float2bfloat16_rn(rem[2 * e + 1]);
      rem[2 * e] -= __bfloat162float(b0);
      rem[2 * e + 1] -= __bfloat162float(b1);
      w[e] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
    }
    *reinterpret_cast<uint4 *>(t0 + p * pstride + o) = make_uint4(w[0], w[1], w[2], w[3]);
  }
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

// One item's operands. K step kt = sh * kc + q reads, for each piece,
//   A: a + sh * a_s + q * a_kt + piece * a_pc   (one 16 KB tile)
//   B: b + sh * b_s + q * b_kt + piece * b_pc   (b_bytes = N rows x 128 B)
// and the rest describes where the epilogue writes.
struct Unit {
  const uint8_t *a, *b;
  int64_t a_kt, a_pc, a_s, b_kt, b_pc, b_s;
  int kc, nk, N;
  uint32_t b_bytes;
  uint8_t *out;              // destination
  int row0, col0;            // destination row / column of accumulator (0, 0)
  int rows, cols;            // valid extent of the destination
  int half[2];               // row-K destinations: K half for the Re / Im rows
  float sgn[2];
  unsigned long long flops;  // algorithmic flops counted for this item (0: none)
};

template <int NMAX, int EPI_SMEM, int P, int SREQ = 3>
struct Ring {
  static constexpr uint32_t A_PIECE = TILE;
  static constexpr uint32_t B_PIECE = NMAX * 128;
  static constexpr uint32_t STAGE = P * (A_PIECE + B_PIECE);
  // SREQ stages, capped at what fits next to the epilogue staging
  static constexpr int S_FIT = (int)((227 * 1024 - 1024 - EPI_SMEM) / STAGE);
  static constexpr int S = S_FIT > SREQ ? SREQ : S_FIT;
  static_assert(S >= 2, "stage ring needs two stages");
  static constexpr int SMEM = 1024 + S * STAGE + EPI_SMEM;
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

// Items blockIdx.x, blockIdx.x + gridDim.x, ... with three roles:
//   warp 4 (one thread): bulk copies of every K step of every item into the
//     stage ring (a stage is refilled once the MMAs that read it completed);
//   warp 5 (one thread): the MMAs of item i into accumulator i % 2, after the
//     epilogue has drained that accumulator (item i - 2);
//   warps 0-3: the epilogue of item i (warp w reads TMEM lanes 32w..32w+31),
//     overlapping the MMAs of item i + 1.
template <class Prob, int NMAX, int SREQ>
__global__ void __launch_bounds__(192, 1) k_cgemm(Prob p, int items, uint32_t *err) {
  constexpr int P = Prob::PIECES;
  using RG = Ring<NMAX, Prob::EPI_SMEM, P, SREQ>;
  constexpr int S = RG::S;
  extern __shared__ uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                            ~(uintptr_t)1023);
  uint8_t *epi_smem = sm + S * RG::STAGE;
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
          tc::mbar_arrive_expect_tx(&full[s], P * (RG::A_PIECE + u.b_bytes));
#pragma unroll
          for (int pc = 0; pc < P; ++pc) {
            tc::bulk_g2s(st + pc * RG::A_PIECE, a + pc * u.a_pc, RG::A_PIECE, &full[s]);
            tc::bulk_g2s(st + P * RG::A_PIECE + pc * RG::B_PIECE, b + pc * u.b_pc, u.b_bytes,
                         &full[s]);
          }
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
          const uint32_t b = a + P * RG::A_PIECE;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // piece products of total order < P, largest first
#pragma unroll
            for (int o = 0; o < P; ++o)
#pragma unroll
              for (int pa = 0; pa <= o; ++pa) {
                const uint64_t ad = tc::smem_desc(a + pa * RG::A_PIECE + j * 256, 128, 1024);
                const uint64_t bd =
                    tc::smem_desc(b + (o - pa) * RG::B_PIECE + j * 256, 128, 1024);
                tc::mma_bf16(d, ad, bd, idesc, (kt > 0 || j > 0 || o > 0) ? 1u : 0u);
              }
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[ab]);
        p.done(u);
        ++n;
      }
      // every MMA issued must have completed before the tensor memory is freed
      tc::mma_commit(&mma_done);
      if (!tc::mbar_wait(&mma_done, 0)) s_fail = 1;
    }
    __syncwarp();
  } else {  // epilogue warps 0-3
    int n = 0;
    for (int it = blockIdx.x; it < items && !*fail; it += gridDim.x) {
      Unit u;
      if (!p.setup(it, u)) continue;
      const int ab = n & 1;
      if (!wait_or_fail(&acc_full[ab], (uint32_t)((n >> 1) & 1), fail)) break;
      tc::fence_after_sync();
      const uint32_t src = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * NMAX);
      for (int c = 0; c < u.N; c += 32) {
        float v[32];
        tc::tmem_ld32(src + (uint32_t)c, v);
        p.epi(u, warp, lane, c, v, epi_smem);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acc_empty[ab]))
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

template <class Prob, int NMAX, int SREQ>
cudaError_t launch_cgemm_s(const Prob &p, int64_t items, uint32_t *err, cudaStream_t s,
                           uint64_t *launches) {
  static int n_sm = 0;
  if (n_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm <= 0)
      n_sm = 1;
  }
  constexpr int SMEM = Ring<NMAX, Prob::EPI_SMEM, Prob::PIECES, SREQ>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_cgemm<Prob, NMAX, SREQ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < n_sm ? items : n_sm);
  k_cgemm<Prob, NMAX, SREQ><<<grid, 192, SMEM, s>>>(p, (int)items, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// stages: requested ring depth (0: as many as fit, at most 3; 2 or 3)
template <class Prob, int NMAX>
cudaError_t launch_cgemm(const Prob &p, int64_t items, uint32_t *err, cudaStream_t s,
                         uint64_t *launches, int stages = 0) {
  if (items <= 0) return cudaSuccess;
  if (items > 0x7fffffff) return cudaErrorInvalidValue;
  if (stages == 2) return launch_cgemm_s<Prob, NMAX, 2>(p, items, err, s, launches);
  return launch_cgemm_s<Prob, NMAX, 3>(p, items, err, s, launches);
}

}  // namespace ctc
