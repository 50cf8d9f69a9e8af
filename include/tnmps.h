/*
 * tnmps.h -- C ABI of the GB300 (sm_103a) matrix-product-state circuit
 * simulator: parameterised-circuit application and Pauli-sum energies.
 *
 * The operations follow arXiv:1807.07914 (McCaskey et al., "Validating
 * Quantum-Classical Programming Models with Tensor Network Simulations"):
 *   - a register of n qubits held as an MPS of n rank-3 tensors (Sec. IV,
 *     ITensor MPS implementation), initialised to a product state;
 *   - single-qubit gates contracted into site tensors and adjacent two-qubit
 *     gates applied by contraction to a rank-4 tensor and an SVD with a
 *     singular-value cutoff (Sec. II, Fig. "mpssvd"; Sec. IV); distant
 *     pairs are joined by SWAP chains (Sec. IV);
 *   - a parameterised circuit executed for runtime parameter values and the
 *     expectation value of every Hamiltonian term per parameter value
 *     (Sec. V.B, VQE), here E(theta) = sum_k c_k <psi(theta)|P_k|psi(theta)>.
 *
 * Conventions
 *   - qubit q lives on MPS site q; bit q of a basis index is qubit q;
 *   - rotations are R_sigma(a) = exp(-i a sigma / 2);
 *   - CNOT: q0 is the control, q1 the target;
 *   - Pauli codes: 1 = X, 2 = Y, 3 = Z.
 *
 * Memory ownership
 *   - The library allocates no device memory. The caller passes a device
 *     arena (sized by tnmps_state_bytes) to tnmps_init and a device
 *     workspace (sized by tnmps_expect_workspace_bytes) to each expectation
 *     call; both must stay valid while the context uses them. Pointers must
 *     be 256-byte aligned.
 *   - Host pointers passed in are read during the call only. Host outputs
 *     are written before the call returns (those calls synchronise the
 *     context's stream). Functions with the suffix _dev take device
 *     pointers, enqueue work on the context's stream and return without
 *     synchronising.
 *
 * Errors
 *   - Every call returns a tnmps_status; no call aborts, exits or traps.
 *     tnmps_last_error(ctx) describes the last failure. Device-side problems
 *     (an SVD that did not converge within its sweep cap, NaN/Inf in the
 *     state, a bounded wait of a tensor-core pipeline that ran out) are
 *     recorded in a device flag and reported by the next synchronising call
 *     or by tnmps_check. After an error the state is unspecified until
 *     tnmps_reset, which also clears the flag; the context stays usable.
 *
 * Threading: a context is used by one host thread at a time.
 */
#ifndef TNMPS_H_INCLUDED
#define TNMPS_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnmps_ctx tnmps_ctx;
typedef struct tnmps_terms tnmps_terms;
typedef struct tnmps_supergate tnmps_supergate;

/* Arithmetic of the state and of the contractions. TNMPS_C128: complex128
 * everywhere (the plain FP64 form). TNMPS_C64: complex64 storage and FP32
 * contractions/rotations; the energy reduction stays FP64.
 * TNMPS_C64_BF16SPLIT: as TNMPS_C64, except that three contractions run on
 * the tensor cores as split-precision complex products, accumulated in FP32:
 *   - the transfer-matrix sweeps of the expectation values, with every FP32
 *     operand value split into two BF16 values hi + lo and each real product
 *     formed as hi*hi + hi*lo + lo*hi (relative rounding of order 2^-16);
 *   - the two-site block of a gate and the right factor U_k^H Theta of its
 *     split, with three BF16 pieces per value (the whole FP32 mantissa, six
 *     piece products), since both feed the state itself.
 * The Jacobi SVD and the orthonormalisation step are those of TNMPS_C64. The
 * state arena holds the converted operands of the tensor-core gate products
 * in addition (tnmps_state_bytes accounts for them). */
typedef enum { TNMPS_C128 = 0, TNMPS_C64 = 1, TNMPS_C64_BF16SPLIT = 2 } tnmps_dtype;

typedef enum {
  TNMPS_OK = 0,
  TNMPS_ERR_ARG = 1,            /* invalid argument or size                   */
  TNMPS_ERR_NOMEM = 2,          /* caller-supplied arena/workspace too small  */
  TNMPS_ERR_UNSUPPORTED = 3,    /* gate or configuration not supported        */
  TNMPS_ERR_NOT_CONVERGED = 4,  /* Jacobi SVD hit its sweep cap               */
  TNMPS_ERR_NUMERIC = 5,        /* NaN or Inf met in singular values/energies */
  TNMPS_ERR_CUDA = 6,           /* a CUDA runtime call failed                 */
  TNMPS_ERR_INJECTED = 7,       /* host-side fault injection (tests only)     */
  TNMPS_ERR_TIMEOUT = 8         /* a device-side wait ran out (a tensor-core
                                   pipeline stalled); the kernel stopped early
                                   and flagged it, its results are invalid      */
} tnmps_status;

/* Gate opcodes (a gate list is the flat form of the paper's IR tree). */
typedef enum {
  TNMPS_I = 0, TNMPS_X = 1, TNMPS_Y = 2, TNMPS_Z = 3, TNMPS_H = 4,
  TNMPS_S = 5, TNMPS_SDG = 6, TNMPS_T = 7,
  TNMPS_RX = 8, TNMPS_RY = 9, TNMPS_RZ = 10,
  TNMPS_CNOT = 16, TNMPS_CZ = 17, TNMPS_SWAP = 18
} tnmps_op;

/* One gate. Rotation angle = angle + scale * theta[param] if param >= 0,
 * else angle (the runtime parameter of Sec. V.B). q1 = -1 for 1q gates. */
typedef struct {
  int32_t op, q0, q1, param;
  double angle, scale;
} tnmps_gate;

/* Counters accumulated since init/reset (for roofline accounting). */
typedef struct {
  uint64_t gates2q;          /* two-qubit gate applications, summed over states */
  uint64_t gates2q_full;     /* ... of which with D_{l-1} = D_l = D_{l+1} = chi_max */
  uint64_t jacobi_pair_rows; /* sum over Jacobi pair visits of the column length */
  uint64_t jacobi_rotations; /* pair visits that rotated                       */
  uint64_t jacobi_sweeps;    /* sweeps, summed over SVDs                       */
  uint64_t svds;             /* SVDs run (states x gates)                      */
  uint64_t env_updates;      /* transfer-matrix updates (nodes x states)       */
  uint64_t env_flops;        /* algorithmic real flops of those updates        */
  uint64_t jacobi_rot_rows;  /* sum over rotated pairs of the column length     */
  uint64_t launches;         /* kernel launches issued by this context (host count) */
  uint64_t jacobi_alg_bytes; /* algorithmic bytes of the SVDs: each block read and
                                written once                                   */
} tnmps_stats;

/* Kernel classes for event timing. */
typedef enum {
  TNMPS_PROF_THETA = 0,   /* two-site block contraction + gate (K2)            */
  TNMPS_PROF_JACOBI = 1,  /* one-sided Jacobi SVD (K3)                          */
  TNMPS_PROF_SPLIT = 2,   /* truncate, orthonormalise, split, normalise (K4)    */
  TNMPS_PROF_MOVE = 3,    /* gauge moves, Householder QR/LQ (K7)                */
  TNMPS_PROF_GATE1 = 4,   /* standalone single-qubit gates (K1)                 */
  TNMPS_PROF_ENV = 5,     /* transfer-matrix environment updates (K5)           */
  TNMPS_PROF_TERM = 6,    /* term values and energy reduction (K6)              */
  TNMPS_PROF_ENV_TC = 7,  /* tensor-core GEMM steps of the K5 sweeps (BF16-split
                             form; nested inside TNMPS_PROF_ENV)                */
  TNMPS_PROF_FIT = 8,     /* super-gate fit contractions: environments and the
                             two-site gradient (its splits count as JACOBI/SPLIT) */
  TNMPS_PROF_SVD_LQ = 9,  /* LQ factorisation of the two-site block ahead of the
                             Jacobi SVD (tnmps_set_svd_precondition mode 1)   */
  TNMPS_PROF_NUM = 10
} tnmps_prof_class;

const char *tnmps_status_string(tnmps_status s);
const char *tnmps_version(void);

/* ---- context ------------------------------------------------------------
 * Device bytes needed for `batch` states of n qubits with bond cap chi_max
 * and up to max_params circuit parameters per state. 0 on bad arguments. */
size_t tnmps_state_bytes(int n_qubits, int chi_max, tnmps_dtype dtype, int batch,
                         int max_params);

/* Create a context on the current CUDA device using `arena` (device memory,
 * arena_bytes >= tnmps_state_bytes(...)). The state is |0...0> for every
 * batch member (Sec. IV: product-state initialisation). Cutoff defaults to
 * 1e-4 (Sec. IV default). 1 <= n_qubits <= 4096, 1 <= chi_max <= 256,
 * batch >= 1. */
tnmps_status tnmps_init(tnmps_ctx **out, int n_qubits, int chi_max, tnmps_dtype dtype,
                        int batch, int max_params, void *arena, size_t arena_bytes);
void tnmps_free(tnmps_ctx *ctx);

/* Singular values sigma_i < eps * ||sigma||_2 are dropped (relative cutoff;
 * the paper's epsilon, Sec. IV); at most chi_max are kept, at least one.
 * The effective cutoff is max(eps, 8u) with u the unit roundoff of the
 * dtype (2^-53 for TNMPS_C128, 2^-24 for TNMPS_C64): singular values at the
 * SVD's rounding-noise floor are always dropped. */
tnmps_status tnmps_set_cutoff(tnmps_ctx *ctx, double eps);
/* Orthogonality tolerance of the Jacobi SVD (Sec. IV's SVD): a column pair
 * counts as orthogonal when |x^H y| <= tol * |x| |y| with
 * tol = factor * (sqrt(rows) + 16) * u (u the dtype's unit roundoff); the
 * iteration ends after the sweep whose largest relative rotation is below
 * sqrt(tol) / 4. factor 1 (default) orthogonalises to the rounding level; a
 * larger factor ends the iteration earlier (fewer sweeps) with the kept
 * singular subspace correspondingly less exact. 1 <= factor <= 4096,
 * TNMPS_ERR_ARG otherwise. */
tnmps_status tnmps_set_svd_tolerance(tnmps_ctx *ctx, double factor);
/* What the Jacobi SVD of a two-site block (Sec. IV) orthogonalises.
 *   mode 1 (default): the block Theta (M x N) is first factored as
 *     Theta = L Q^H (Householder QR of Theta^H, Q not formed) and the Jacobi
 *     runs on the columns of the lower-trapezoidal L (M x min(M, N)). Theta
 *     and L have the same singular values and left singular vectors, and the
 *     split forms U_k^H Theta from Theta itself, so the result is the same SVD;
 *     L's columns start closer to orthogonal (their Gram matrix is one
 *     QR-iteration step past Theta Theta^H), so fewer sweeps are needed.
 *   mode 0: the Jacobi runs on the columns of Theta.
 * TNMPS_ERR_ARG on any other mode. */
tnmps_status tnmps_set_svd_precondition(tnmps_ctx *ctx, int mode);
/* CUDA stream (cudaStream_t) for all work of this context; NULL = default. */
tnmps_status tnmps_set_stream(tnmps_ctx *ctx, void *stream);
/* Back to |0...0> with zero discarded weight and zeroed counters. */
tnmps_status tnmps_reset(tnmps_ctx *ctx);

/* ---- circuits ------------------------------------------------------------
 * Apply a gate list to every state. theta: host array [n_params] shared by
 * all states. Two-qubit gates on distant qubits use SWAP chains. */
tnmps_status tnmps_apply_circuit(tnmps_ctx *ctx, const tnmps_gate *gates, size_t n_gates,
                                 const double *theta, size_t n_params);
/* Same, one parameter row per state: thetas host array [batch][n_params]. */
tnmps_status tnmps_apply_circuit_batched(tnmps_ctx *ctx, const tnmps_gate *gates,
                                         size_t n_gates, const double *thetas,
                                         size_t n_params);
/* Same, thetas a device array [batch][n_params]; asynchronous. */
tnmps_status tnmps_apply_circuit_batched_dev(tnmps_ctx *ctx, const tnmps_gate *gates,
                                             size_t n_gates, const double *thetas_dev,
                                             size_t n_params);

/* ---- Pauli sums -----------------------------------------------------------
 * A term set in CSR form: term k acts with paulis[j] on sites[j] for
 * term_off[k] <= j < term_off[k+1]; coeffs[k] is real. A term with no sites
 * is the identity. Sites within a term must be distinct and < n_qubits.
 * The host builds the prefix trie of the terms once here; arrays are copied. */
tnmps_status tnmps_terms_create(tnmps_terms **out, int n_qubits, const int32_t *term_off,
                                const int32_t *sites, const uint8_t *paulis,
                                const double *coeffs, size_t n_terms);
void tnmps_terms_free(tnmps_terms *terms);
/* Trie size: nodes (= transfer updates per state), depth, widest level. */
tnmps_status tnmps_terms_info(const tnmps_terms *terms, int64_t *n_nodes, int32_t *depth,
                              int64_t *max_level_nodes);
/* Device workspace bytes for evaluating `terms` on ctx with states processed
 * in chunks of theta_chunk (0 = the whole batch at once). */
size_t tnmps_expect_workspace_bytes(const tnmps_ctx *ctx, const tnmps_terms *terms,
                                    int theta_chunk);
/* E[b] = sum_k c_k <psi_b|P_k|psi_b> for every state b (host outputs,
 * energy[batch]; per_term[batch][n_terms] of Re<P_k> may be NULL). */
tnmps_status tnmps_expect_pauli_sum(tnmps_ctx *ctx, const tnmps_terms *terms, void *ws,
                                    size_t ws_bytes, double *energy, double *per_term);
/* Same with device outputs; asynchronous. */
tnmps_status tnmps_expect_pauli_sum_dev(tnmps_ctx *ctx, const tnmps_terms *terms, void *ws,
                                        size_t ws_bytes, double *energy_dev,
                                        double *per_term_dev);

/* ---- measurement ----------------------------------------------------------
 * Shots of a computational-basis measurement of every qubit (the MEASURE
 * instructions that end the kernels of Sec. V.B), sampled exactly: qubits
 * n-1, n-2, ..., 0 in turn, each drawn from its probability conditioned on
 * the outcomes already drawn for the qubits above it.
 *   uniforms_dev: device FP64 [batch][shots][n_qubits], values in [0, 1),
 *     caller-owned, read during the call's GPU work. uniforms[b][k][q]
 *     decides qubit q of shot k of state b: outcome 0 iff it is below
 *     P(q = 0 | outcomes above q) (computed in FP64 from the state's
 *     arithmetic type).
 *   bits_dev: device uint8 [batch][shots][n_qubits], written 0 or 1.
 * Moves the orthogonality centre to site n-1, as the energy calls do;
 * allocates nothing; asynchronous on the context's stream.
 * Errors: TNMPS_ERR_ARG (null pointer, shots < 1); a zero-norm state raises
 * TNMPS_ERR_NUMERIC at the next synchronising call. */
tnmps_status tnmps_sample_dev(tnmps_ctx *ctx, const double *uniforms_dev, int shots,
                              uint8_t *bits_dev);

/* ---- super-gates by overlap maximisation ----------------------------------
 * The general gate action of Sec. II (steps 1-6) and of Sec. IV's ExaTENSOR
 * MPS visitor: an ordered aggregate of gates on any qubits (a super-gate) is
 * applied by optimising an output MPS TN_out so that the closed network
 * <TN_out | gates . TN_inp> is as large as possible.
 *
 * tnmps_supergate_create: gates as for tnmps_apply_circuit (any distance
 * between the qubits of a two-qubit gate), parameters bound from theta[n_params]
 * (host, read during the call). The host builds the gates as a matrix-product
 * operator over the window [first, last] of qubits they touch (two-qubit
 * gates through an exact operator-Schmidt split, bonds reduced to the ranks of
 * the operator's cuts, at most 64). TNMPS_ERR_ARG on a bad gate,
 * TNMPS_ERR_UNSUPPORTED if an MPO bond would exceed 64. No device work. */
tnmps_status tnmps_supergate_create(tnmps_supergate **out, int n_qubits, const tnmps_gate *gates,
                                    size_t n_gates, const double *theta, size_t n_params);
void tnmps_supergate_free(tnmps_supergate *sg);
/* Window and MPO bonds: bonds[last - first + 2], bonds[0] = bonds[end] = 1
 * (either pointer may be NULL). */
tnmps_status tnmps_supergate_info(const tnmps_supergate *sg, int32_t *first, int32_t *last,
                                  int32_t *bonds);
/* The MPO tensors, site first..last in order, each [w_left][2 out][2 in]
 * [w_right] row-major, as interleaved complex128 (cap = doubles available;
 * TNMPS_ERR_NOMEM if too small). */
tnmps_status tnmps_supergate_mpo(const tnmps_supergate *sg, double *out, size_t cap);
/* Device workspace bytes of tnmps_apply_supergate for this context (0 on a
 * mismatch of register sizes). */
size_t tnmps_supergate_workspace_bytes(const tnmps_ctx *ctx, const tnmps_supergate *sg);
/* Apply the super-gate to every state of the context. Stages: (3) TN_out is
 * a copy of the state, first brought to the gates applied one by one
 * (adjacent pairs, SWAP chains, truncation under the stage's bond cap);
 * (5) left-to-right sweeps of two-site updates over the window, each update
 * the normalised gradient of the overlap with respect to the two-site block,
 * split by the SVD and the cutoff rule under the bond cap, until no state's
 * fidelity F = |<TN_out|gates TN_inp>|^2 rises by tol in a sweep (or
 * max_sweeps); (6) while some state has 1 - F > target and the cap is below
 * chi_max (<= the context's chi_max), the cap (initially the largest bond of
 * the input inside the window) doubles and the stage repeats from the copy.
 * Sites outside the window keep the input's tensors. The discarded weight of
 * each state grows by 1 - F.
 *   ws: device workspace of tnmps_supergate_workspace_bytes (256-byte
 *       aligned), caller-owned.
 *   fidelity[batch], fidelity_start[batch] (F of the last stage's first
 *   iterate), info[3] = {sweeps, stages, final bond cap}: host outputs, each
 *   may be NULL. Synchronises the context's stream (one read of the
 *   overlaps per sweep). */
tnmps_status tnmps_apply_supergate(tnmps_ctx *ctx, const tnmps_supergate *sg, int chi_max,
                                   double target, double tol, int max_sweeps, void *ws,
                                   size_t ws_bytes, double *fidelity, double *fidelity_start,
                                   int32_t *info);

/* ---- inspection ------------------------------------------------------------ */
/* Synchronise and report device-side error flags. */
tnmps_status tnmps_check(tnmps_ctx *ctx);
/* Bond dimensions: dims[batch][n_qubits - 1] (synchronises). */
tnmps_status tnmps_get_bond_dims(tnmps_ctx *ctx, int32_t *dims);
/* Cumulative discarded weight per state: w[batch] (synchronises). */
tnmps_status tnmps_get_discarded_weight(tnmps_ctx *ctx, double *w);
/* Copy site tensor `site` of state b to host as complex128 (re, im pairs),
 * row-major (D_{site-1}, 2, D_site); `cap` = capacity in complex elements. */
tnmps_status tnmps_get_site(tnmps_ctx *ctx, int b, int site, double *out, size_t cap,
                            int32_t *dl, int32_t *dr);
/* Orthogonality centre (site index) after the work enqueued so far. */
int tnmps_get_centre(const tnmps_ctx *ctx);
tnmps_status tnmps_get_stats(tnmps_ctx *ctx, tnmps_stats *out);
/* ---- launch shapes (autotuning) ---------------------------------------------
 * Runtime choices of launch shape for the hot kernels of a context; every
 * choice computes the same results (up to FP32 summation order), only the
 * speed differs. An autotuner times the choices on the caller's workload and
 * sets the fastest. The paper has no counterpart (its simulator was serial).
 *   jacobi_shape[c]: the complex64 Jacobi SVD for blocks of up to 64, 128,
 *     256 rows (c = 0, 1, 2):
 *       0 (default) c = 0, 1: one CTA of 512 threads per SM, 32-column blocks;
 *                   c = 2: two CTAs of 256 threads per SM, 16-column blocks;
 *       1           c = 0, 1: two CTAs of 256 threads per SM, 16-column blocks;
 *                   c = 2: one CTA of 512 threads per SM, 32-column blocks.
 *     (complex128 and blocks above 256 rows have a single shape.)
 *   gemm_stages: shared-memory ring depth of the tensor-core GEMMs of the
 *     BF16-split form (two-site block, split, sweeps): 0 (default) = as many
 *     as fit, at most 3; or 2 or 3 (capped at what fits).
 *   sweep_fused: transfer sweeps of the BF16-split form: 0 (default) = each
 *     trie level as two launches (all step-1 products, then all step-2
 *     products, the intermediates in the workspace); 1 = one launch per level
 *     whose CTAs run both steps of their own (state, node) updates, the
 *     intermediates in two slots per CTA that stay in L2.
 * TNMPS_ERR_ARG on any other value. */
typedef struct {
  int32_t jacobi_shape[3];
  int32_t gemm_stages;
  int32_t sweep_fused;
} tnmps_tuning;
tnmps_status tnmps_set_tuning(tnmps_ctx *ctx, const tnmps_tuning *tuning);
tnmps_status tnmps_get_tuning(const tnmps_ctx *ctx, tnmps_tuning *tuning);

/* Time the kernel classes in class_mask (bit i = tnmps_prof_class i) with
 * CUDA events recorded on the context's stream around each launch group;
 * totals are cleared. class_mask = 0 stops timing. */
tnmps_status tnmps_profile(tnmps_ctx *ctx, uint32_t class_mask);
/* Synchronise and return accumulated milliseconds and launch-group counts
 * per class (arrays of TNMPS_PROF_NUM entries, either may be NULL). */
tnmps_status tnmps_profile_read(tnmps_ctx *ctx, double *ms, uint64_t *count);
const char *tnmps_last_error(const tnmps_ctx *ctx);

/* ---- standalone kernels (unit parity) --------------------------------------
 * One-sided Jacobi SVD (the gate step's SVD, Sec. IV) on `batch` column-major
 * m x n matrices: a_dev points to batch*lda*n complex elements (complex128
 * or complex64 per dtype; matrix b at a_dev + b*lda*n). On return the
 * columns are mutually orthogonal (A V); sigma_dev[batch][n] receives the
 * column norms (unsorted) and sweeps_dev[batch] the sweep counts.
 * m <= 512, n <= 512, lda >= m. Asynchronous on `stream`. */
tnmps_status tnmps_jacobi_svd_dev(tnmps_dtype dtype, int batch, int m, int n, void *a_dev,
                                  int lda, double *sigma_dev, int32_t *sweeps_dev,
                                  int max_sweeps, void *stream);

/* ---- ALU ceiling (measurement) ---------------------------------------------
 * The paper has no counterpart: this measures the issue rate of fused
 * multiply-adds on the CUDA cores, the ceiling of the ALU-bound Jacobi SVD,
 * so that its roofline fraction is taken against a measured rate. One launch
 * of `blocks` CTAs of 256 threads; every thread runs 8 independent FMA
 * chains for 64 * iters FMAs, in FP32 (bits = 32) or FP64 (bits = 64).
 *   sink_dev: device buffer of blocks * 256 elements of that type (written);
 *   *flops (may be NULL): floating-point operations of the launch
 *     (2 per FMA).
 * The caller times the launch (CUDA events on `stream`); asynchronous.
 * TNMPS_ERR_ARG on bits not 32/64, blocks or iters < 1, or a NULL sink. */
tnmps_status tnmps_alu_peak_dev(int bits, int blocks, int iters, void *sink_dev, double *flops,
                                void *stream);

/* ---- many circuits in one persistent launch --------------------------------
 * Independent jobs with uneven register sizes, depths, bond caps and Pauli
 * sums (the VQE loop of Sec. V.B run for many programs at once), complex64
 * state and FP64 energies. One kernel launch runs every job: each CTA pulls
 * whole jobs, most expensive first, and simulates them end to end.
 * All job arrays are host memory, read by tnmps_batch_create only. */
typedef struct {
  int32_t n_qubits;           /* 2..256                                     */
  int32_t chi_max;            /* 1..128                                     */
  const tnmps_gate *gates;    /* gate list (as tnmps_apply_circuit)         */
  int32_t n_gates;
  const double *theta;        /* [n_params]                                 */
  int32_t n_params;
  const int32_t *term_off;    /* Pauli sum in CSR form (as tnmps_terms_create) */
  const int32_t *sites;
  const uint8_t *paulis;
  const double *coeffs;
  int32_t n_terms;
} tnmps_job;
typedef struct tnmps_batch tnmps_batch;
/* Plan every job on the host (gate fusion, gauge moves, term tries). */
tnmps_status tnmps_batch_create(tnmps_batch **out, const tnmps_job *jobs, int n_jobs,
                                double cutoff);
/* Device bytes for `ctas` persistent CTAs (one scratch slice each). */
size_t tnmps_batch_bytes(const tnmps_batch *batch, int ctas);
/* Upload the plan into `arena` (synchronous) and fix the launch shape:
 * `ctas` CTAs of 256 threads, Jacobi column blocks of 16 or 32. */
tnmps_status tnmps_batch_bind(tnmps_batch *batch, void *arena, size_t bytes, int ctas,
                              int block_cols, void *stream);
/* Capture the launch (work-counter reset + kernel) as a CUDA graph; later
 * tnmps_batch_launch calls replay it. */
tnmps_status tnmps_batch_capture_graph(tnmps_batch *batch);
/* Enqueue the whole batch (asynchronous). */
tnmps_status tnmps_batch_launch(tnmps_batch *batch);
/* Synchronise; energies[n_jobs] (and per-job discarded weight, may be NULL). */
tnmps_status tnmps_batch_results(tnmps_batch *batch, double *energy, double *discarded);
tnmps_status tnmps_batch_info(const tnmps_batch *batch, int64_t *n_ops, int64_t *n_nodes,
                              double *est_cost);
const char *tnmps_batch_last_error(const tnmps_batch *batch);
void tnmps_batch_free(tnmps_batch *batch);

/* ---- energies without any device allocation --------------------------------
 * For callers that cannot call cudaMalloc -- code that runs under a device
 * memory budget a host framework has already reserved in full, or a loop
 * that must never enter the allocator. Same results and arguments as
 * tnmps_expect_pauli_sum_dev without the workspace: the library uses its own
 * scratch, a static device array of TNMPS_NOALLOC_SCRATCH_BYTES (160 MiB: one
 * state of a 40-qubit, chi = 128 register with a 157-term Heisenberg chain
 * needs about 100 MB in the BF16-split form and 127 MB in complex128) that
 * every GPU loading the library holds until the process exits. The paper has
 * no counterpart to this entry point.
 *   - The first call on a device looks up the array's device address for the
 *     current CUDA context (and again whenever the context changes, e.g.
 *     after cudaDeviceReset); make that first call before any stream capture.
 *   - Term sets (with this context) needing more scratch than the array
 *     holds for a single state are rejected with TNMPS_ERR_NOMEM and a
 *     message giving both sizes. States are processed in chunks that fit;
 *     the per-term region is reserved only when per_term_dev is NULL.
 *   - All calls share the array, which keeps the last call's contents. The
 *     term plan is uploaded (from host memory; this synchronises the
 *     context's stream) when the array last held another context's or
 *     another term set's plan; a repeated call with the same context and
 *     term set is asynchronous on the context's stream. Calls whose GPU
 *     work overlaps -- other streams, other contexts, other host threads --
 *     race on the array.
 *   - Allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *     call. */
#define TNMPS_NOALLOC_SCRATCH_BYTES (160u << 20)
tnmps_status tnmps_expect_pauli_sum_noalloc(tnmps_ctx *ctx, const tnmps_terms *terms,
                                            double *energy_dev, double *per_term_dev);

/* BF16 GEMM on the tensor cores (tcgen05, FP32 accumulation in tensor memory):
 * C[M x N] = A[M x K] * B[N x K]^T with A, B given as BF16 bit patterns
 * (uint16), both K-major (row r of A at A + r*lda), C row-major FP32.
 * K, lda, ldb multiples of 8; A, B 16-byte aligned. Asynchronous on
 * `stream`. Used by the surrogate's layers; exported for unit parity (this
 * entry point has no context flag: a bounded wait that runs out leaves C
 * undefined without a report; the surrogate's own calls report it through
 * tnmps_mlp_check). */
tnmps_status tnmps_gemm_bf16_dev(int M, int N, int K, const uint16_t *A, int lda,
                                 const uint16_t *B, int ldb, float *C, int ldc, void *stream);

/* ---- learned surrogate of E(theta) -----------------------------------------
 * MLP d_in -> width -> width -> 1 with SiLU (d_in, width multiples of 8),
 * FP32 master weights, BF16 GEMMs on the tensor cores with FP32
 * accumulation, last layer, elementwise work and Adam in FP32. The paper has
 * no learned component; the surrogate proposes optimiser steps for the VQE
 * loop of Sec. V.B and the MPS simulation verifies them. Parameters are a
 * flat FP32 vector: W1 (width x d_in, row-major), b1, W2 (width x width),
 * b2, w3 (width), b3. All pointers are device pointers; all calls are
 * asynchronous on the surrogate's stream (tnmps_mlp_set_stream). */
typedef struct tnmps_mlp tnmps_mlp;
size_t tnmps_mlp_bytes(int d_in, int width, int max_batch);
int64_t tnmps_mlp_num_params(int d_in, int width);
tnmps_status tnmps_mlp_init(tnmps_mlp **out, int d_in, int width, int max_batch, void *arena,
                            size_t arena_bytes);
void tnmps_mlp_free(tnmps_mlp *mlp);
tnmps_status tnmps_mlp_set_stream(tnmps_mlp *mlp, void *stream);
const char *tnmps_mlp_last_error(const tnmps_mlp *mlp);
/* Synchronise the surrogate's stream and report its device flag: a bounded
 * wait of a tensor-core GEMM that ran out gives TNMPS_ERR_TIMEOUT (the flag
 * is cleared; the results since the last check are invalid). */
tnmps_status tnmps_mlp_check(tnmps_mlp *mlp);
/* copy parameters in (also clears the Adam moments) / out */
tnmps_status tnmps_mlp_set_params(tnmps_mlp *mlp, const float *params_dev);
tnmps_status tnmps_mlp_get_params(tnmps_mlp *mlp, float *params_dev);
/* y[B] = f(x[B][d_in]) */
tnmps_status tnmps_mlp_forward(tnmps_mlp *mlp, const float *x_dev, int B, float *y_dev);
/* Forward + backward. With targets: loss = mean (y - t)^2 and its gradients;
 * without (target_dev NULL): gradients of sum_b y_b, so grad_x[b] = dy_b/dx_b
 * (the surrogate's gradient of E). Any output pointer may be NULL. */
tnmps_status tnmps_mlp_backward(tnmps_mlp *mlp, const float *x_dev, const float *target_dev,
                                int B, float *y_dev, float *loss_dev, float *grad_params_dev,
                                float *grad_x_dev);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step counts from 1) on
 * the MSE loss of the batch. */
tnmps_status tnmps_mlp_train_step(tnmps_mlp *mlp, const float *x_dev, const float *target_dev,
                                  int B, float lr, int step, float *loss_dev);

/* Failure-detection test of the device-side waits (no paper counterpart):
 * enqueues one kernel that waits on an mbarrier phase that nothing completes,
 * with a limit of max_cycles SM clocks (1 <= max_cycles <= 2^31); when the
 * wait runs out it raises the context's timeout flag and returns, exactly as
 * a stalled tensor-core pipeline does. The next synchronising call reports
 * TNMPS_ERR_TIMEOUT; tnmps_reset clears it. Asynchronous on the context's
 * stream; never faults or hangs the GPU. */
tnmps_status tnmps_debug_wait_timeout(tnmps_ctx *ctx, int64_t max_cycles);

/* Host-side fault injection for error-path tests: the call number `nth`
 * (counting from 1) of any state-changing entry point returns `status`
 * before touching the device. nth = 0 disarms. */
tnmps_status tnmps_debug_inject(tnmps_ctx *ctx, int nth, tnmps_status status);

#ifdef __cplusplus
}
#endif
#endif /* TNMPS_H_INCLUDED */
