/*
 * rsvd_mlp.h -- the rank-prediction network and its probe features.
 *
 * The paper chooses the rank R_SVD and the oversampling p by hand
 * ("Randomized matrix decompositions" paragraph: l = R_SVD + p, p = 5).  This
 * library adds a small learned model that predicts, per channel and
 * tolerance, the rank and oversampling from a cheap probe sketch, so that one
 * fixed-rank pass replaces the blocks of the adaptive loop; the adaptive loop
 * remains its fallback, and the rank rule's error check decides whether a
 * predicted rank is accepted (RSVD_RANK_LEARNED in rsvd.h).
 *
 * Network: x (d) -> tanh(x W1 + b1) (128) -> tanh(. W2 + b2) (128) -> . W3 + b3 (2),
 * outputs (log k, log p).  Parameter blob (FP32, device, caller-owned), row-major:
 *   W1 (d x 128) | b1 (128) | W2 (128 x 128) | b2 (128) | W3 (128 x 2) | b3 (2).
 * Loss: mean over batch and outputs of (y - t)^2.  Adam: Kingma & Ba, ICLR 2015.
 *
 * Features (d = RSVD_MLP_FEATURES = 19) of a channel from the 16-column probe
 * Y16 = V P16 (P16: Philox stream tag 1, the plan's seed):
 *   log(t_j / t_1), j = 2..16  (t = singular values of Y16, floored at 1e-300)
 *   log t_1, 0.5 log(||Y16||_F^2 / 16), log n, log tol.
 *
 * All pointers are DEVICE pointers unless stated; every call is asynchronous
 * on `stream` (cudaStream_t, NULL = legacy default) and returns
 * RSVD_ERR_INVALID_ARG for bad sizes or NULL pointers without launching.
 */
#ifndef RSVD_MLP_H
#define RSVD_MLP_H

#include "rsvd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RSVD_MLP_HIDDEN 128
#define RSVD_MLP_FEATURES 19

/* Number of FP32 parameters for input width d. */
int64_t rsvd_mlp_param_count(int32_t d);

/* Floats of caller-owned scratch rsvd_mlp_loss_grad needs for batch B. */
int64_t rsvd_mlp_work_floats(int32_t d, int32_t B);

/* Y (B x 2, row-major) = network(X (B x d, row-major)). */
rsvd_status rsvd_mlp_forward(const float* theta, int32_t d, const float* X, int32_t B, float* Y,
                             void* stream);

/* grad (param blob layout) = d loss / d theta on the batch (X, T (B x 2));
 * *loss (device float) = the loss.  work: rsvd_mlp_work_floats(d, B) floats. */
rsvd_status rsvd_mlp_loss_grad(const float* theta, int32_t d, const float* X, const float* T, int32_t B,
                               float* grad, float* loss, float* work, void* stream);

/* One Adam step on nparams parameters; t >= 1 is the step count. */
rsvd_status rsvd_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t nparams, int32_t t,
                          float lr, float beta1, float beta2, float eps, void* stream);

/* Standardisation of training data: mean and sd (device, d floats each) of
 * the columns of X (N x d, row-major), sums in FP64, the population standard
 * deviation floored at sd_floor (> 0); Xn (N x d) = (X - mean) / sd.  Used
 * on the features and on the targets before training. */
rsvd_status rsvd_mlp_standardize(const float* X, int32_t N, int32_t d, float sd_floor, float* mean, float* sd,
                                 float* Xn, void* stream);

/* Fold the standardisation into a network trained on standardised data, so
 * that `out` (a separate blob of the same size) takes raw features and gives
 * raw targets: W1 / sd_x, b1 - (mean_x / sd_x) W1, W3 sd_t, b3 sd_t + mean_t. */
rsvd_status rsvd_mlp_fold(const float* theta, int32_t d, const float* mean_x, const float* sd_x,
                          const float* mean_t, const float* sd_t, float* out, void* stream);

/* Minibatch gather: dst[r, :] = src[idx[r], :] for r < B, rows of `cols`
 * floats (idx: B int64 row numbers on the device, drawn by the caller). */
rsvd_status rsvd_mlp_gather_rows(const float* src, const int64_t* idx, int32_t B, int32_t cols, float* dst,
                                 void* stream);

/* Probe features of C channels (FP32, C x RSVD_MLP_FEATURES row-major, device)
 * using the plan's precision and seed; tol: host array of C tolerances.
 * Synchronous. */
rsvd_status rsvd_probe_features(rsvd_plan_t plan, int32_t C, const rsvd_matrix* A, const double* tol,
                                float* features);

#ifdef __cplusplus
}
#endif
#endif /* RSVD_MLP_H */
