// Internal launcher declarations of the rSVD CUDA kernels (not part of the ABI).
#pragma once

#include "common.cuh"

namespace rsvd {

// Count of kernels launched by the library (benchmark accounting).
void note_launch(int k = 1);
long long launch_count();

// ----------------------------------------------------------------- tile GEMMs
enum MMMode { MM_STORE = 0, MM_ATOMIC = 1, MM_PARTIAL = 2, MM_SUB = 4 };
// MM_SUB: C <- C - A B (block Gram-Schmidt against earlier blocks).
enum MMKind {
  MMK_DENSE_F64 = 0,     // C = V B, V dense row-major FP64, FP64 FMA
  MMK_GRAM_F64 = 1,      // partial C_s = Y_s^T Z_s, FP64
  MMK_NN_F64 = 2,        // C = A B, A tall column-major FP64
  MMK_GRAM_DOT2 = 3,     // partial C_s = Y_s^T Z_s, FP32 data, compensated (Dot2) -> FP64
  MMK_NN_F32_F64B = 4,   // C(FP32) = A(FP32) B(FP64 rounded to FP32), FP32 FMA
  MMK_NN_F32_OUT64 = 5,  // C(FP64) = A(FP32) B(FP64 rounded to FP32), FP32 FMA
  MMK_GRAM_F32 = 6,      // partial C_s = Y_s^T Z_s, FP32 data, FP32 FMA -> FP64 partials
  MMK_NN_F32 = 7,        // C(FP32) = A(FP32) B(FP32), FP32 FMA
  MMK_NN_F32_OUT64_B32 = 8   // C(FP64) = A(FP32) B(FP32), FP32 FMA
};

struct MMDesc {
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  void* Cm; int64_t ldc;
  int m, n, k;
  int mt, nt, ks, kchunk;   // tiles along m, n; k splits and their length
  int mode;                 // MMMode
  int sym;                  // Gram: only upper tiles
  int64_t pstride;          // MM_PARTIAL: elements between split partials
  const double* colscale;   // optional per-output-column scale
  __nv_bfloat16* sl[3];     // optional BF16 slices of the result (column-major, ldsl)
  int64_t ldsl;
  int nsl;
  const int* ncols_dev;     // optional: output columns limited to *ncols_dev (rank chosen on device)
  int tile;                 // output tile edge of the kernel kind (64 or 128)
  const int* cond;          // optional: run only if (*cond & FLAG_SHIFTED) (a conditional CholeskyQR round)
};

int tile_of(MMKind kind);

struct ZeroDesc { void* p; int64_t ld; int rows, cols, esz; };
void launch_zero(const ZeroDesc* d_zd, const int* d_off, int C, int tiles, cudaStream_t st);

void launch_tile_mm(MMKind kind, const MMDesc* d_md, const int* d_off, int C, int tiles,
                    cudaStream_t st);
void launch_reduce_partials(const MMDesc* d_md, double* const* d_out, int C, int max_elems,
                            cudaStream_t st);

// Tensor-core Gram G = Y^T Y of an FP32 panel (mixed path, l <= 128) to
// FP64-grade accuracy: per channel the panel (column-major, ldy a multiple of
// 4, 16-byte aligned), the workspace of its 128-row tiles (gram_tc_part_floats
// floats, 128 ints per tile) and the FP64 output (l x l, leading dim l, both
// triangles).  Two launches; returns a cudaError_t value.
struct GramTcDesc {
  const float* Y; int64_t ldy;
  int n, l;
  int tile0, ntiles;        // first tile of the channel in the launch, its tile count
  float* part;              // ntiles x {hi, lo} x 128 x 128
  int* exps;                // ntiles x 128 column exponents
  double* G;
};
// fp32_grade: three slices and the exact products of levels 2-4 only.
int launch_gram_tc(const GramTcDesc* d_gd, int C, int tiles, int fp32_grade, int* d_err, cudaStream_t st);
int gram_tc_part_floats(int n);

// Tensor-core product C = A B of a tall FP32 panel A (n x K, K <= 128,
// column-major lda) and a small B (K x N, N <= 128, FP32 or FP64 (b64),
// column-major ldb, columns optionally scaled by colscale): C32 (FP32, with
// nsl BF16 words into sl) or C64 (FP64), leading dim ldc; columns from
// *ncols_dev on are not written; channels with cond set and the shifted
// flag clear are skipped.  bimg (nn_tc_img_bytes(), 16-byte aligned) and
// fexp (128 ints) are per-channel scratch.  Two launches.
struct NnTcDesc {
  const float* A; int64_t lda;
  int n, K, N;
  int tile0;
  const void* B; int64_t ldb;
  int b64;
  const double* colscale;
  void* bimg;
  int* fexp;
  float* C32;
  double* C64;
  int64_t ldc;
  __nv_bfloat16* sl[3];
  int64_t ldsl;
  int nsl;
  const int* ncols_dev;
  const int* cond;
};
int launch_nn_tc(const NnTcDesc* d_nd, int C, int tiles, int* d_err, cudaStream_t st);
int nn_tc_img_bytes();

// Probe block of the mixed path (s <= 32, l <= 256): C = Q^T Z over row
// splits (partials, then their sum, FP64 C, leading dim l), then Z -= Q C.
// Two descriptor arrays with the same channels: in d_tn, tile0 is the
// channel's first block of the C = Q^T Z launch (splits x ceil(l / 128)
// blocks each), in d_nn its first block of the Z -= Q C launch
// (ceil(n / 128) blocks each).
struct ProbeDesc {
  const float* Q; int64_t ldq;
  float* Z; int64_t ldz;
  int n, l, s;
  int tile0;
  int splits, split_rows;
  double* part;
  double* C;
  float* C32;               // C rounded to FP32, l rows of 32 (16-byte aligned, l * 32 floats)
};
void launch_probe_block(const ProbeDesc* d_tn, const ProbeDesc* d_nn, int C, int tn_blocks, int nn_blocks,
                        cudaStream_t st);

// ------------------------------------------------------------ small kernels
// ||A||_F^2 partials per 64-row block, non-finite detection (dense input).
void launch_fro2(const Chan* d_ch, const int* d_off_rows64, int C, int tiles, cudaStream_t st);
void launch_fro2_reduce(const Chan* d_ch, int C, cudaStream_t st);
void launch_fro2_reduce_rows(const Chan* d_ch, int C, int rows_per_part, cudaStream_t st);
// Omega (FP64 form) into X[:, 0:l) of each channel, columns col0 + j.
void launch_omega_f64(const Chan* d_ch, const int* d_off, int C, int tiles, uint64_t seed,
                      int col0, cudaStream_t st, uint32_t tag = TAG_OMEGA);
// Upper Cholesky G = R^T R (l x l), R^{-1}; R_acc <- R R_acc when accumulate.
// Shifted retry on breakdown (flag FLAG_SHIFTED).
// conditional: only channels whose result flags carry FLAG_SHIFTED.
void launch_chol_inv(const Chan* d_ch, int C, int accumulate, int max_l, int f32_inverse,
                     cudaStream_t st, int f32_chol = 0, int conditional = 0);
// Q32 <- T32 (n x l) for channels whose result flags carry FLAG_SHIFTED.
void launch_copy_t_to_q_if_shifted(const Chan* d_ch, int C, cudaStream_t st);
// dst <- src (count doubles) for channels whose *flags carries FLAG_SHIFTED.
struct CopyDesc { const double* src; double* dst; int64_t count; const int* flags; };
void launch_copy64_if_shifted(const CopyDesc* d_cd, int C, cudaStream_t st);
// One-sided Jacobi SVD of M = R^T (FP64 or FP32 arithmetic); writes sig, M <- left
// vectors, J <- right vectors, sorted by descending sigma.
void launch_jacobi(const Chan* d_ch, int C, int fp32, int max_l, cudaStream_t st);
// The same on a cooperative grid, several CTAs per channel (for l past the
// single CTA's shared memory); h_l: host copy of the channels' l.  coop_ws:
// kCoopWsInts zero-able ints of device scratch.  Returns 0, or -1 if it did
// not launch (the caller then runs launch_jacobi).
constexpr int kCoopMaxChannels = 512;
constexpr int kCoopWsInts = 4 + 60 * kCoopMaxChannels;
// Controls of the cooperative kernels' grid barriers and of the Jacobi sweep
// cap.  err: the plan's device error word (DERR_TIMEOUT_BARRIER when a
// barrier wait expires; the call then returns RSVD_ERR_TIMEOUT).  budget:
// clocks one barrier wait may spin (default 2^32, about two seconds).
// stall: test hook, CTA 0 never arrives, so the other CTAs' waits expire.
// max_sweeps: Jacobi sweep cap (default 60; reaching it with pairs still
// rotating gives RSVD_ERR_NOT_CONVERGED).  coop_ctl fills them from the
// environment: RSVD_WAIT_CLOCKS, RSVD_TEST_STALL_BARRIER (1 = on),
// RSVD_JACOBI_MAX_SWEEPS (1..60) -- diagnostics for tests.
struct CoopCtl { int* err; long long budget; int stall; int max_sweeps; };
CoopCtl coop_ctl(int* err);
int jacobi_max_sweeps();
int launch_jacobi_coop(const Chan* d_ch, const int* h_l, int C, int fp32, int* coop_ws, int* err, cudaStream_t st);
// Cholesky + inverse (launch_chol_inv's contract, FP64 inverse) on a
// cooperative grid; same return convention.
int launch_chol_coop(const Chan* d_ch, const int* h_l, int C, int accumulate, int f32_chol, int conditional,
                     int* coop_ws, int* err, cudaStream_t st);
// Rank selection (fixed or tolerance) from sig and ||A||^2 (FP64 identity),
// or from the probe residual (mixed path).  Writes S and ChanResult.
// Probe rule: with s Gaussian probe columns g_j the energies
// e_j(k) = ||(I - U_k U_k^T) V g_j||^2 are i.i.d. with mean ||(I - U_k U_k^T) V||_F^2.
// A rank is accepted when the upper confidence bound  mean + PROBE_Z sd / sqrt(s)
// (sd the sample deviation of the e_j) is at most tol^2 ||V||_F^2.  With
// s = 32 probes PROBE_Z is a little above the one-sided 99.9% point of
// Student's t with 31 degrees of freedom (3.37), leaving room for the skew of
// the e_j (weighted chi-square sums).  The reported estimate is the mean.
constexpr double PROBE_Z = 3.5;
// Energy the probe estimate cannot see on the mixed path: the remainder the
// BF16 words leave out of V (measured while converting) plus the FP32
// rounding of the lifted factors, modelled as 2 sqrt(l) eps_32 relative.
// Both the rank rule and the adaptive stop add it to the estimate.
__host__ __device__ inline double precision_floor2(double wres2, int l, double fro2) {
  return wres2 + 4.0 * l * 3.552713678800501e-15 * fro2;     // eps_32^2 = 2^-48
}
void launch_select(const Chan* d_ch, int C, int policy, double tol, int use_probe,
                   cudaStream_t st);
// Sign fix: largest-|.| entry of U_i positive, flip V_i with it.
void launch_signfix(const Chan* d_ch, int C, int max_k, cudaStream_t st);
// out[c] = sum of squares of the n x cols block at p[c] (leading dim ld[c]), FP64.
struct SumsqDesc { const void* p; int64_t ld; int rows, cols, esz; double* out; };
void launch_sumsq(const SumsqDesc* d_sd, int C, cudaStream_t st);
// out[c][j] = sum of squares of column j of the block (one block per column).
void launch_colsumsq(const SumsqDesc* d_sd, int C, int max_cols, cudaStream_t st);

// --------------------------------------------------------------- tile rule
// H (n x M, ldh) = sqrt(w_m) g_m(x_j), scaled by hscale (a power of two that
// puts max H at 2^14), as two FP16 words of its FP32 value.
struct RuleDesc {
  int n, M;
  const double *c, *s, *w;   // device, M each
  __half* H[2];
  int64_t ldh;
  double hscale;
};
// The power of two hscale for the rule weights (max sqrt(w_m) to 2^14).
double rule_hscale(const double* w, int M);
// Re-orthonormalisation steps of the FP32 Jacobi vectors (l <= 128): 0 scale
// the Gram of M by D on both sides, 1 Ri32 = D (R^{-1} - I), 2 J += M D.
void launch_reorth(int stage, const Chan* d_ch, int C, int max_l, cudaStream_t st);
struct CvtDesc { const double* src; float* dst; int64_t count; };
void launch_cvt_f32(const CvtDesc* d_desc, int C, int64_t max_count, cudaStream_t st);
void launch_sym_signs(const double* U, int64_t ldu, const double* V, int64_t ldv, int n, int k, double* signs,
                      cudaStream_t st);
void launch_rule_prep(const RuleDesc& d, cudaStream_t st);
// FP64 path: the factor panel in FP64, and the noise (+ energy partials) of a
// generated FP64 row panel (kRuleNoiseBlocks pairs in part).
struct RuleDesc64 {
  int n, M;
  const double *c, *s, *w;   // device, M each
  double* H;
  int64_t ldh;
};
constexpr int kRuleNoiseBlocks = 1216;
void launch_rule_prep64(const RuleDesc64& d, cudaStream_t st);
void launch_rule_noise64(double* P, int64_t ldp, int rows, int n, int r0, uint32_t key, double amp3, double* part,
                         cudaStream_t st);
void launch_rule_part_sum(const double* part, int nparts, double* out, cudaStream_t st);
void launch_rule_finish(const double* sums, int npanels, ChanResult* res, cudaStream_t st);

// --------------------------------------------------------- mixed-path kernels
void launch_convert_slices(const Chan* d_ch, const int* d_off_rows, int C, int tiles, int nsl,
                           cudaStream_t st);
void launch_omega_bf16(const Chan* d_ch, const int* d_off, int C, int tiles, uint64_t seed,
                       int col0, int j0, int j1, uint64_t pseed, int nsl, cudaStream_t st,
                       uint32_t tag = TAG_OMEGA);
// launch_convert_slices and the full launch_omega_bf16 (col0 = 0, all columns,
// TAG_OMEGA) as one interleaved grid.
void launch_convert_omega(const Chan* d_ch, const int* d_off8, int t8, const int* d_off64, int t64, int C, int nsl,
                          uint64_t seed, uint64_t pseed, int onsl, cudaStream_t st);
// 19 rank-model features per channel from its probe singular values (h.sig).
void launch_features(const Chan* d_ch, int C, double tol, float* feat, cudaStream_t st);
void launch_probe_finish(const Chan* d_ch, int C, int max_l, cudaStream_t st);

// ------------------------------------------------------------ exact residual
// Both write resid_blocks(n) partial pairs {residual^2, ||A||^2} to part.
// A is read column-major (A[r + c lda]).  The rule form regenerates every
// entry in FP64: H (n x ldh, row j contiguous over m) from launch_rule_prep64
// plus the hash noise (amp3 = noise scale * sqrt(3)).
int resid_blocks(int64_t n);
void launch_resid(const double* A, int64_t lda, const double* U, int64_t ldu, const double* V, int64_t ldv,
                  const double* S, int n, int k, double* part, cudaStream_t st);
void launch_resid_rule(const double* H, int64_t ldh, int M, uint32_t key, double amp3, const double* U,
                       int64_t ldu, const double* V, int64_t ldv, const double* S, int n, int k, double* part,
                       cudaStream_t st);

// Error text of the calling thread (rsvd_last_error_string) for entry points
// outside the plan code: clear it on entry, set it with a failure.
void clear_error_text();
rsvd_status set_error_text(rsvd_status s, const char* fmt, ...);

}  // namespace rsvd
