/*
 * rsvd.h -- C ABI of the GB300 randomized low-rank decomposition library.
 *
 * Problem statement (arXiv:2307.15572, "Randomized matrix decompositions"
 * paragraph, Eq. (1) and Fig. 1): given a dense matrix V (N x N) -- here a
 * symmetric channel block of an interaction -- and either a target rank
 * R_SVD with oversampling p = l - R_SVD, or a relative tolerance, return
 * the leading singular triplets  V ~ L_k Sigma_k R_k^T.  The method is the
 * randomized SVD the paper takes from Halko, Martinsson & Tropp (2011):
 *   1. Z = V P with a random P (N x l); orthonormal Q with Z = Q X;
 *      optional subspace iteration (q rounds, re-orthogonalised);
 *   2. Y = Q^T V and its thin SVD  Y = L_Y Sigma R^T;
 *   3. L = Q L_Y.
 * Channels of a block-diagonal matrix ("Low-rank interactions" paragraph:
 * one block per J^Pi T channel, sizes 7650..40050) are independent and are
 * decomposed together by rsvd_decompose_batched.
 *
 * Conventions shared by every entry point:
 *   - Plain C types only; every pointer argument says whether it is a host or
 *     a device pointer.  Dense matrices are FP64.  Because V is symmetric,
 *     row-major and column-major storage coincide; `ld` is the distance in
 *     elements between consecutive rows (= columns), ld >= n.
 *   - Factors are column-major: U[i + j*ldu] is row i of column j.
 *   - The caller owns all input and output buffers.  The plan owns its
 *     device workspace (allocated with cudaMalloc when the plan is created
 *     or first needs more; freed by rsvd_plan_destroy).
 *   - Errors are returned as rsvd_status; no C++ exception crosses this ABI.
 *     rsvd_last_error_string() gives a thread-local description of the last
 *     failure.  Negative = error, 0 = OK, positive = warning (result valid).
 *   - Input is never modified.  Work runs on the plan's CUDA stream; the
 *     decomposition calls return after that stream has finished the work
 *     (they read the chosen rank and status words back), so outputs are
 *     ready when they return.
 */
#ifndef RSVD_H
#define RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSVD_OK = 0,
  RSVD_WARN_SHIFTED_CQR = 1,    /* a Cholesky breakdown was repaired by a shift  */
  RSVD_WARN_RANK_CAPPED = 2,    /* l = k + p was clamped to n                      */
  RSVD_ERR_INVALID_ARG = -1,    /* bad size, pointer, enum or leading dimension    */
  RSVD_ERR_CUDA = -2,           /* a CUDA runtime/driver call failed               */
  RSVD_ERR_OOM = -3,            /* workspace allocation failed                     */
  RSVD_ERR_NONFINITE = -4,      /* NaN or Inf found in the input                   */
  RSVD_ERR_NOT_CONVERGED = -5,  /* Jacobi sweep cap reached                        */
  RSVD_ERR_TOL_NOT_MET = -6,    /* tolerance not reached within l_max columns;
                                   the best factors found are still returned      */
  RSVD_ERR_TIMEOUT = -7,        /* a bounded device-side wait gave up              */
  RSVD_ERR_UNSUPPORTED = -8     /* combination not built (reported, never faked)   */
} rsvd_status;

/* Arithmetic of the passes over V. */
typedef enum {
  RSVD_PREC_FP64 = 0,   /* every step in FP64 (CUDA cores); the accuracy reference path */
  RSVD_PREC_BF16X = 1   /* V split into `slices` BF16 words, tcgen05 tensor-core passes
                           with FP32 accumulation; FP64 Gram/Cholesky (compensated)      */
} rsvd_precision;

/* How the rank is chosen. */
typedef enum {
  RSVD_RANK_FIXED = 0,    /* R_SVD = k, l = k + p (paper's setting)                      */
  RSVD_RANK_TOL = 1,      /* l = k + p columns drawn, R_SVD = smallest rank meeting tol  */
  RSVD_RANK_ADAPTIVE = 2, /* blocks of block_b columns until tol is met (randQB_EI)      */
  RSVD_RANK_LEARNED = 3   /* per-channel l from the rank model, checked, adaptive fallback */
} rsvd_rank_policy;
/* ADAPTIVE stops a channel once its error indicator is under tol (or l_max
 * columns are drawn).  FP64: the exact indicator ||V||^2 - sum ||B_i||^2.
 * BF16X: that difference cancels at the passes' precision, so the indicator
 * comes from 32 Gaussian probe columns g_j: the energies ||(I - Q Q^T) V g_j||^2,
 * kept up to date block by block, whose mean estimates the squared error.
 * A channel stops (and a rank is accepted, in TOL mode too) when an upper
 * confidence bound (mean + 3.5 standard errors), plus the precision floor of
 * the BF16 words and the FP32 factors, is under tol^2 ||V||_F^2.
 * LEARNED falls back to ADAPTIVE in the plan's own precision. */

typedef struct {
  int64_t n_max;        /* largest channel size the plan will be given (>= 1)            */
  int32_t k;            /* FIXED: rank R_SVD; TOL/LEARNED: cap on the rank (0 = l)       */
  int32_t p;            /* oversampling p = l - R_SVD (>= 0; paper uses 5)               */
  int32_t q;            /* subspace-iteration rounds (>= 0; paper uses 0)                */
  double tol;           /* relative Frobenius tolerance for TOL/ADAPTIVE/LEARNED (> 0)  */
  int32_t l_max;        /* cap on columns drawn (ADAPTIVE/LEARNED fallback; 0 = 1024)    */
  int32_t block_b;      /* ADAPTIVE block size (0 = 32)                                   */
  int32_t precision;    /* rsvd_precision                                                 */
  int32_t slices;       /* BF16X: BF16 words per FP64 entry for the passes (1..3; 0 = 2) */
  int32_t rank_policy;  /* rsvd_rank_policy                                               */
  int32_t rayleigh_ritz;/* 1: symmetric Rayleigh-Ritz small problem (T = Q^T V Q)         */
  uint64_t seed;        /* Philox key of the random projection P                          */
  void* stream;         /* cudaStream_t to run on (NULL = legacy default stream)          */
  const float* mlp_weights; /* LEARNED: device pointer to the rank-model parameter blob   */
} rsvd_opts;

typedef struct rsvd_plan_s* rsvd_plan_t;

typedef enum {
  RSVD_DENSE_F64 = 0,   /* stored matrix                                            */
  RSVD_TILE_RULE = 1    /* entries from the Gaussian-bump rule, generated on device */
} rsvd_matrix_kind;

typedef enum { RSVD_MEM_DEVICE = 0, RSVD_MEM_HOST = 1 } rsvd_mem;

/*
 * A channel matrix.  DENSE_F64: `data` is an n x n symmetric FP64 matrix with
 * leading dimension ld >= n, in device memory (mem = DEVICE) or host memory
 * (mem = HOST; page-locked memory gives overlapped copies).  The library
 * does not check symmetry.
 * TILE_RULE: entries A_ij = sum_m w_m g_m(x_i) g_m(x_j) + eta_ij with
 * x_i = 8 i/(n-1), g_m(x) = exp(-(x-c_m)^2/(2 s_m^2)) (1 <= rule_m <= 4096,
 * s_m > 0, w_m >= 0) and eta the symmetric hash noise of standard deviation
 * rule_eta keyed by rule_seed:
 *   h = mix(mix(min(i,j) * 0x9E3779B1 + key) ^ (max(i,j) * 0x85EBCA77)),
 *   eta_ij = rule_eta sqrt(3) (2 u - 1), u = ((h >> 8) + 1/2) 2^-24,
 *   key = mix(seed_lo ^ mix(seed_hi)), mix = the 32-bit "lowbias32" hash
 * (arithmetic modulo 2^32).  rule_c, rule_s, rule_w are HOST arrays of
 * rule_m values; `data`, `ld` and `mem` are ignored.  The matrix is never
 * stored: every pass generates the entries it reads, row panel by row panel:
 * with precision BF16X on the tensor core (the factor sqrt(w_m) g_m(x_j) as
 * two FP16 words scaled by a power of two, three word products, FP32
 * accumulation; entries accurate to ~1e-6 relative), with precision FP64 on
 * the CUDA cores in FP64 (2 rule_m FP64 flops per entry and pass).  Any rank
 * policy (the adaptive loop generates the matrix 2 + 2q times per block of
 * block_b columns).  Tile rules cannot share a call with stored channels
 * (RSVD_ERR_UNSUPPORTED otherwise).  Tuning: the environment variable
 * RSVD_RULE_PANEL sets the rows generated per panel (default: panels of
 * ~8 GiB of words).
 */
typedef struct {
  int32_t kind;
  int32_t mem;
  int64_t n;
  const double* data;
  int64_t ld;
  int32_t rule_m;
  const double* rule_c;
  const double* rule_s;
  const double* rule_w;
  double rule_eta;
  uint64_t rule_seed;
} rsvd_matrix;

/*
 * Output factors of one channel, caller-owned.  U (n x k_cap, ldu >= n),
 * V (n x k_cap, ldv >= n) and S (k_cap) are FP64, in device memory
 * (mem = DEVICE) or host memory (mem = HOST).  Any of U, V may be NULL to
 * skip it.  On return: k_out = rank kept (<= k_cap; singular values in S
 * are descending and the pair (U_i, V_i) is sign-fixed so that the
 * largest-magnitude entry of U_i is positive), l_used = columns drawn,
 * err_est = estimated relative Frobenius error of the rank-k_out factors,
 * status = this channel's rsvd_status.  `tol` (input) overrides the plan's
 * tolerance for this channel when > 0.
 */
typedef struct {
  int32_t mem;
  double* U;
  int64_t ldu;
  double* S;
  double* V;
  int64_t ldv;
  int32_t k_cap;
  int32_t k_out;
  int32_t l_used;
  double err_est;
  int32_t status;
  double tol;           /* input: this channel's tolerance (0 = the plan's), TOL/ADAPTIVE/LEARNED */
} rsvd_factors;

/* Create a plan.  Checks the options (RSVD_ERR_INVALID_ARG on a bad value)
 * and allocates the fixed part of the device workspace.  *out is NULL on
 * failure. */
rsvd_status rsvd_plan(rsvd_plan_t* out, const rsvd_opts* opts);

/* Free the plan and its workspace.  NULL is ignored. */
void rsvd_plan_destroy(rsvd_plan_t plan);

/* Decompose one channel: equivalent to rsvd_decompose_batched with C = 1. */
rsvd_status rsvd_decompose(rsvd_plan_t plan, const rsvd_matrix* A, rsvd_factors* f);

/* Decompose C independent channels (C >= 1) of possibly different sizes in
 * grouped launches: every kernel of the pipeline covers all channels at once.
 * per_item (host, C entries, may be NULL) receives each channel's status,
 * which is also stored in f[c].status.  Returns the worst status (the most
 * negative error if any, else the largest warning, else RSVD_OK). */
rsvd_status rsvd_decompose_batched(rsvd_plan_t plan, int32_t C, const rsvd_matrix* A,
                                   rsvd_factors* f, rsvd_status* per_item);

/* Exact relative residual ||A - U diag(S) V^T||_F / ||A||_F of the rank-f->k_out
 * factors, accumulated in FP64 over every entry (the paper's validation of
 * a rank-R_SVD form, "Randomized matrix decompositions" paragraph).  Stored
 * channels (device or host A and factors) are read as they are.  Tile rules
 * are regenerated: every entry is rebuilt in FP64 from the rule's definition
 * (the FP64 factor panel sqrt(w_m) g_m(x_j), its products and the hash
 * noise) and compared with the factors tile by tile, nothing of A being
 * stored -- 2 n^2 (rule_m + k) FP64 flops, e.g. about a minute at
 * n = 200,000 on this part's FP64 rate.  For A = 0 the absolute residual
 * ||U diag(S) V^T||_F is returned.  *rel_err is a host pointer; synchronous.
 * The plan's workspace grows by n * rule_m doubles for a tile rule. */
rsvd_status rsvd_reconstruct_error(rsvd_plan_t plan, const rsvd_matrix* A,
                                   const rsvd_factors* f, double* rel_err);

/* Launch accounting of the plan's own kernels, for benchmarks.  When enabled
 * (rsvd_plan_set_profiling(plan, 1)), each decomposition records CUDA events
 * on the plan's stream around every tensor-core pass, every FP64 dense pass
 * over V, every tile-rule generation, every conversion of V into words and
 * every tensor-core Gram of CholeskyQR, every tensor-core tall x small
 * product and every pass reading FP64 V directly, and adds their device time and algorithmic traffic (bytes of V words, X
 * words and Y read or written once, as the roofline counts them) to the
 * counters below.  Kernel launches are counted whether or not timing is
 * enabled.  rsvd_plan_profile copies the counters (host struct) and, if
 * `reset` is non-zero, zeroes them. */
typedef struct {
  int64_t launches;        /* kernels launched by this plan                     */
  int64_t tc_launches;     /* tensor-core passes over V                          */
  double tc_ms;            /* their summed device time (CUDA events)             */
  double tc_bytes;         /* their summed algorithmic bytes                     */
  double tc_flops;         /* their summed MMA flops (2 m n k per word pair)     */
  int64_t f64_launches;    /* FP64 dense passes over V                           */
  double f64_ms;
  double f64_flops;        /* 2 n^2 l per pass                                   */
  int64_t gen_launches;    /* tile-rule generation launches (one per row panel)  */
  double gen_ms;
  double gen_flops;        /* algorithmic: 2 M per generated entry               */
  double gen_mma_flops;    /* issued: 3 word products x 2 x (M padded to 64)     */
  int64_t cvt_launches;    /* conversions of stored FP64 V into BF16 words       */
  double cvt_ms;
  double cvt_bytes;        /* 8 B read + 2 B per word written per entry          */
  int64_t gram_launches;   /* tensor-core Grams Y^T Y of n x l FP32 panels        */
  double gram_ms;          /* (both kernels: slice products and tile reduction)  */
  double gram_flops;       /* algorithmic: 2 n l^2 per Gram                      */
  double gram_mma_flops;   /* issued: 21 slice products x 2 x 128^3 per tile     */
  int64_t nn_launches;     /* tensor-core tall x small products (Y R^-1, lifts)   */
  double nn_ms;
  double nn_flops;         /* algorithmic: 2 n l N per product                   */
  int64_t f64in_launches;  /* tensor-core passes reading stored FP64 V directly  */
  double f64in_ms;
  double f64in_bytes;      /* 8 B per V entry, + X words and Y once              */
  double f64in_flops;      /* MMA flops (2 n^2 N per word pair)                  */
} rsvd_profile;

rsvd_status rsvd_plan_set_profiling(rsvd_plan_t plan, int32_t enable);

/* CUDA graphs (off by default).  When enabled, and the plan's stream is not
 * the legacy default stream and profiling is off, each fixed/tolerance/learned
 * decomposition -- stored channels or tile rules -- is captured once per
 * shape (channel sizes, options, the plan's buffers and staged host inputs;
 * for tile rules also rule_m, rule_seed, rule_eta and the scale of the
 * weights) and replayed on later calls of the same shape; device input and
 * output pointers and the rule's centres, widths and weights may change
 * between replays.  Up to 8 graphs are kept (least recently used evicted);
 * growing the workspace drops them.  The adaptive loop is not captured (it
 * synchronises per block).  Disabling frees the graphs. */
rsvd_status rsvd_plan_set_graphs(rsvd_plan_t plan, int32_t enable);
rsvd_status rsvd_plan_profile(rsvd_plan_t plan, rsvd_profile* out, int32_t reset);

/* Autotuning of launch shapes (off by default).
 *
 * The grouped passes over the channels (Fig. 1 steps 1 and 2 and the power
 * iterations: the tensor-core products of the mixed path and the FP64
 * products of the FP64 path) can be launched in several shapes that compute
 * the same result up to the order of FP32/FP64 summation: the output-column
 * tile width, the k-split policy (how many work items per SM the split aims
 * for, and the shortest split), the shared-memory pipeline depth, and the
 * order in which the persistent CTAs take the channels' work items.  With
 * autotuning on, the first execution of a pass whose signature (kind of pass,
 * word counts, every channel's size and column count) this plan has not seen
 * times every distinct candidate shape on the caller's own data -- one
 * warm-up launch, then the better of two timed launches each -- keeps the
 * fastest (the fixed default rule unless another is at least 2% faster) and
 * runs it; later passes with that signature, in the same call and in later
 * calls, run the chosen shape without timing.  A call that tunes synchronises
 * its stream between candidates and is not captured into a CUDA graph (later
 * calls of the same shape are, if graphs are on).  Enabling drops the plan's
 * captured graphs; disabling keeps the choices already made (the plan keeps
 * using them) and stops tuning new signatures.  The tile-rule passes keep
 * their fixed shapes.  rsvd_plan_tune_records copies up to `cap` records of
 * the choices, in the order they were made, and sets *count to the number
 * the plan holds.  For diagnostics, the environment variable
 * RSVD_TUNE_FORCE=i makes every new signature take candidate i (modulo the
 * number of candidates) after timing them. */
enum { RSVD_TUNE_TC = 0, RSVD_TUNE_DENSE_F64 = 1 };
typedef struct {
  int32_t kind;            /* RSVD_TUNE_TC or RSVD_TUNE_DENSE_F64                 */
  int32_t candidates;      /* distinct shapes timed                              */
  int32_t choice;          /* index of the chosen shape (0: the default rule)    */
  int32_t bn;              /* output-column tile width                           */
  int32_t split_target;    /* work items the k split aims for (0: no split)      */
  int32_t min_split;       /* shortest k split, rows of V                        */
  int32_t stages;          /* shared-memory pipeline stages (tensor-core pass)   */
  int32_t order;           /* 1: longest channel first, 0: channel order         */
  float ms_default;        /* device time of the default shape (best of two)    */
  float ms_best;           /* device time of the chosen shape                    */
  float tune_ms;           /* host time spent tuning this signature              */
} rsvd_tune_record;

rsvd_status rsvd_plan_set_autotune(rsvd_plan_t plan, int32_t enable);
rsvd_status rsvd_plan_tune_records(rsvd_plan_t plan, rsvd_tune_record* out, int32_t cap, int32_t* count);

/* Basis transformation on the thin factors ("Low-rank interactions"
 * paragraph, after Eq. (3): V-bar = U^dagger V U operates only on the thin
 * L and R^dagger).  For factors f of an n x n channel (DEVICE buffers,
 * k = f->k_out) and a basis B (n x m, DEVICE, column-major, ldb >= n; any B,
 * not only unitary), writes Lt = B^T U_k (m x k, ldl >= m) and
 * Rt = B^T V_k (m x k, ldr >= m), FP64, so that
 *   B^T V B ~ Lt diag(S) Rt^T
 * at 4 m n k flops instead of the 2 n^2 m + 2 n m^2 of transforming V.
 * Runs on the plan's stream (its workspace holds two descriptors) and
 * returns after the stream has completed.  RSVD_ERR_INVALID_ARG for host
 * factors, bad sizes or pointers; k = 0 writes nothing. */
rsvd_status rsvd_transform_factors(rsvd_plan_t plan, const rsvd_factors* f, int64_t n, const double* B,
                                   int64_t ldb, int64_t m, double* Lt, int64_t ldl, double* Rt, int64_t ldr);

/* FP64-grade Gram G = Y^T Y of an FP32 panel: the Gram of CholeskyQR
 * (Fukaya, Nakatsukasa, Yanagisawa & Yamamoto, 2014), which orthonormalises
 * the sketch Y = A Omega of the paper's step 1 and factors W^T W of the
 * projection on the mixed path.  Y (DEVICE, n x l FP32, column-major,
 * ldy >= n) and G (DEVICE, l x l FP64, column-major, leading dim l, both
 * triangles written).
 *   method RSVD_GRAM_TC: tensor cores; each 128-row tile of Y is split into
 *     six exact BF16 fixed-point slices (Ozaki, Ogita, Oishi & Rump, 2012),
 *     the leading slice products summed exactly in TMEM and the tiles in
 *     double-float.  Needs l <= 128, ldy a multiple of 4 and Y 16-byte
 *     aligned.
 *   method RSVD_GRAM_TC_F32: the same with three slices and only the exact
 *     products (the Gram of Y rounded to 24 fractional bits of its tile-
 *     column maxima): FP32-grade, for a Y that is already nearly
 *     orthonormal (CholeskyQR's second round).
 *   method RSVD_GRAM_DOT2: CUDA cores, compensated dot products (Ogita,
 *     Rump & Oishi, 2005), any l.
 * RSVD_GRAM_TC and RSVD_GRAM_DOT2 agree with the exact Gram of the FP32 data
 * to about 1e-13 of ||y_i|| ||y_j||, RSVD_GRAM_TC_F32 to about 2^-23.  The decompositions of the mixed path use RSVD_GRAM_TC
 * where every channel has l <= 128 (unless the environment variable
 * RSVD_GRAM=dot2 is set when the call is built).  Uses the plan's workspace
 * and stream and returns after the stream has completed.
 * RSVD_ERR_INVALID_ARG for NULL pointers, n < 1, l < 1, ldy < n or a bad
 * method; RSVD_ERR_UNSUPPORTED for a tensor-core method with l > 128 or a
 * misaligned Y; RSVD_ERR_TIMEOUT if a bounded device wait expired. */
enum { RSVD_GRAM_TC = 0, RSVD_GRAM_DOT2 = 1, RSVD_GRAM_TC_F32 = 2 };
rsvd_status rsvd_gram_f32(rsvd_plan_t plan, const float* Y, int64_t ldy, int64_t n, int32_t l, double* G,
                          int32_t method);

/* Tall x small product C = A B on the tensor cores, FP32-grade: the product
 * behind CholeskyQR's Q = Y R^{-1} and the lifts U = Q X, V = W X Sigma^{-1}
 * of the paper's step 3 on the mixed path.  A (DEVICE, n x K FP32,
 * column-major, lda >= n), B (DEVICE, K x N, FP64 if b_fp64 else FP32,
 * column-major, ldb >= K), C (DEVICE, n x N, FP64 if c_fp64 else FP32,
 * column-major, ldc >= n), 1 <= K, N <= 128.  Each row of A and each column
 * of B is split into three 8-bit fixed-point BF16 slices (after a power-of-
 * two scaling), the slice products summed exactly in TMEM: C is the exact
 * product of A and B rounded to 24 fractional bits of their row (column)
 * maxima, rounded once to FP32 (C FP64: that FP32 value, widened).  Uses the
 * plan's workspace and stream and returns after the stream has completed.
 * RSVD_ERR_INVALID_ARG for NULL pointers or bad sizes, RSVD_ERR_UNSUPPORTED
 * for K or N above 128, RSVD_ERR_TIMEOUT if a bounded device wait expired. */
rsvd_status rsvd_panel_product(rsvd_plan_t plan, const float* A, int64_t lda, int64_t n, int32_t K, const void* B,
                               int64_t ldb, int32_t b_fp64, int32_t N, void* C, int64_t ldc, int32_t c_fp64);

/* Symmetric storage.  For symmetric V the singular triplets pair as
 * v_i = sign(lambda_i) u_i (lambda_i the eigenvalue of magnitude sigma_i), so
 * V ~ U_k diag(sign_i sigma_i) U_k^T: only U_k, S and the k signs need to be
 * kept, which is the one-factor reading of the compression ratio below.
 * signs (DEVICE, k doubles) receives sign(u_i . v_i) = +-1 for the factors f
 * of an n x n channel (DEVICE buffers); asynchronous on the plan's stream. */
rsvd_status rsvd_symmetric_signs(rsvd_plan_t plan, const rsvd_factors* f, int64_t n, double* signs);

/* Compression ratio of a rank-k form of an n x n matrix (the paper's
 * compression-ratio equation in "Randomized matrix decompositions"):
 * one_factor = 0: n^2 / (2 n k + k) as printed (both factors stored);
 * one_factor = 1: n^2 / (n k + k) (symmetric storage: U_k and S, signs
 * folded in), the reading under which a relative rank of 1 % gives C ~ 100
 * as the text states.  Returns 0 for n < 1 or k < 1. */
double rsvd_compression_ratio(int64_t n, int32_t k, int32_t one_factor);

/* Exact relative residual with no device allocation (no plan needed).
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory when they check a decomposition -- callers whose
 * device memory is fully reserved up front by their own pool (a further
 * cudaMalloc would fail or break their budget), and callers that must not let
 * cudaMalloc/cudaFree synchronise the device in the middle of a pipeline.
 * It computes the same quantity as rsvd_reconstruct_error,
 * ||A - U diag(S) V^T||_F / ||A||_F in FP64, but keeps its per-tile partial
 * sums in a fixed array of 2 x 1,216 doubles (19 KiB) that the library holds
 * on every GPU that loads it, until the process exits.
 *
 *   A (n x n, leading dim lda >= n; any matrix, read column-major
 *   A[r + c*lda]), U (n x k, ldu >= n), S (k), V (n x k, ldv >= n): DEVICE
 *   pointers, column-major as elsewhere;
 *   rel_err: DEVICE pointer to one double, written asynchronously (for A = 0
 *   the absolute residual ||U diag(S) V^T||_F);
 *   stream: cudaStream_t (NULL = legacy default stream).
 * n is limited to RSVD_NOALLOC_MAX_N.  Returns RSVD_ERR_INVALID_ARG for
 * n < 1, n > RSVD_NOALLOC_MAX_N, k < 0 or a bad pointer or leading dimension
 * (nothing is launched then), RSVD_ERR_CUDA if a CUDA call fails; the reason
 * is in rsvd_last_error_string().  It calls no cudaMalloc, cudaFree or
 * allocating library routine.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before capturing any stream on the device, and do not
 * call the entry point again after a cudaDeviceReset in the same process
 * (the looked-up address belonged to the old context).  All calls on one
 * device share the array, so calls that overlap on the GPU (concurrent
 * streams, or several host threads) race and must be serialised by the
 * caller. */
#define RSVD_NOALLOC_MAX_N 16384
rsvd_status rsvd_reconstruct_error_noalloc(const double* A, int64_t lda, int64_t n, const double* U,
                                           int64_t ldu, const double* S, const double* V, int64_t ldv,
                                           int32_t k, double* rel_err, void* stream);

/* Rows r0 .. r0+rows-1 of a tile rule as the decomposition's passes generate
 * them (FP32, noise included, before the split into BF16 words):
 * out[p * ldo + j] = A_(r0+p, j), out a DEVICE pointer, ldo >= n.  Uses the
 * plan's stream and workspace (grown if needed); synchronous.  Returns
 * RSVD_ERR_INVALID_ARG for a matrix that is not a tile rule, bad parameters
 * or rows outside [0, n). */
rsvd_status rsvd_rule_rows(rsvd_plan_t plan, const rsvd_matrix* A, int64_t r0, int32_t rows, float* out,
                           int64_t ldo);

/* Device buffer size (bytes) the plan holds now. */
int64_t rsvd_plan_workspace_bytes(rsvd_plan_t plan);

/* Thread-local text of the last error ("" if none). */
const char* rsvd_last_error_string(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t rsvd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RSVD_H */
