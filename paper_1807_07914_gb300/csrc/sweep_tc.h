// Host interface of the tensor-core transfer sweeps (dtype
// TNMPS_C64_BF16SPLIT): buffer geometry and the per-level launchers.
#pragma once
#include "tnmps_internal.h"

namespace swtc {

// One operand tile: 128 rows x 64 BF16 of K, canonical no-swizzle K-major
// layout of 8-row x 16-byte core matrices (byte offset of (r, k) =
// (r/8)*1024 + (k/8)*128 + (r%8)*16 + (k%8)*2).
constexpr int TILE = 16384;
// Complex K values per tile: the Re parts fill K 0..31, the Im parts 32..63.
constexpr int KCH = 32;

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Row-K matrix (environment, or one s-half of the intermediate T) of up to
// chi rows and chi complex columns, tiles ordered [K chunk][piece hi/lo][row
// tile]: the first r rows of every row tile of one (chunk, piece) are one
// contiguous run of r * 128 bytes.
inline int64_t rowk_bytes(int chi) {
  return (int64_t)cdiv(chi, KCH) * 2 * cdiv(chi, 128) * TILE;
}
// Converted operands of one site with bond capacities (cl, cr): the
// real-embedded X^T (2 * ceil(cr/64) row tiles) and X_0^H, X_1^H
// (ceil(cr/64) row tiles each), over ceil(cl/32) K chunks, hi and lo.
inline int64_t site_bytes(int cl, int cr) {
  return (int64_t)8 * cdiv(cl, KCH) * cdiv(cr, 64) * TILE;
}

}  // namespace swtc

struct TcSweep {
  const int32_t *dims;      // StateView dims, [batch][n+1]
  int n, b0, nb;            // states b0 .. b0+nb-1 of the context
  uint8_t *site_ops;        // [nb][site_stride]
  const int64_t *site_off;  // device [n]: byte offset of site i inside one state's block
  const int32_t *site_geo;  // device [n][2]: {ceil(cap_l/32), ceil(cap_r/64)}
  int64_t site_stride;
  uint8_t *lprev, *lcur;    // [level nodes][nb][env_bytes]
  uint8_t *tbuf;            // [level nodes][nb][2][env_bytes]
  int64_t env_bytes;
  int rt;                   // row tiles of an environment (ceil(chi/128))
  int nmax;                 // 128 or 256: widest MMA N (>= every bond dimension)
  int stages;               // GEMM ring depth request (0: as many as fit)
  int fused;                // 1: both steps of a level in one launch (k_sweep_fused)
  int64_t tslots;           // (state, node) T buffers in tbuf (each 2 x env_bytes)
  uint32_t *err;
};

// Convert every site tensor of the chunk's states into the two A operands.
cudaError_t tc_prep_sites(const TcSweep &t, const void *sites, const int64_t *site_off_elems,
                          int64_t state_elems, cudaStream_t s, uint64_t *launches);
// Identity environments in lprev for the first trie level (root nodes).
cudaError_t tc_root_envs(const TcSweep &t, const int32_t *node_site, int nodes, int dmax,
                         cudaStream_t s, uint64_t *launches);
// One trie level: T = L_parent (P X), then L = X^H T, for every (node, state).
// level1: the parent of node k is the identity environment at lprev slot k.
cudaError_t tc_level(const TcSweep &t, const int32_t *node_site, const int32_t *node_parent,
                     const int32_t *node_pauli, int nodes, bool level1, int dmax_r,
                     unsigned long long *counters, cudaStream_t s, uint64_t *launches);
// <P_t> = Re sum_{c,c'} L[c][c'] R[c][c'] for the terms that end on this level.
cudaError_t tc_term_dot(const TcSweep &t, const void *renv, const int64_t *roff,
                        int64_t renv_elems, const int32_t *tterm, const int32_t *tnode,
                        const int32_t *tsite, int count, int64_t n_terms, double *per_term,
                        cudaStream_t s, uint64_t *launches);
