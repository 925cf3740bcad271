/*
 * sur.h — C ABI of the surrogate network trained on the ensemble solver's output.
 *
 * Not part of the paper: its uncertainty propagation runs the ensemble solver directly
 * (Section 1, Section 3). This library adds a learned shortcut for repeated statistics:
 * a multilayer perceptron n_in -> H -> H -> n_out with GELU activations maps the
 * truncated Karhunen-Loeve coefficients of the realisation's E and h fields to POD
 * coefficients of a displacement field the solver produced. Training minimises the mean
 * squared error with Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8). Matrix products run
 * on the fifth-generation tensor cores (tcgen05, accumulator in tensor memory) in BF16
 * with FP32 accumulation; parameters, activations, gradients and optimiser state are FP32.
 * The products wait for the tensor cores with bounded waits; one that gives up is reported
 * as SUR_ERR_CUDA by the next call that synchronises (sur_loss_grad, sur_loss, sur_train).
 *
 * Conventions: every call returns SUR_OK (0) or a negative SUR_ERR_* code and
 * sur_last_error gives the message. Arrays with the suffix _dev are device pointers
 * (row-major, FP32, caller-owned); host arrays are caller-owned. Work runs on the stream
 * given to sur_create and calls that return host data synchronise it.
 * Parameter vector layout (sur_get_params, sur_set_params, gradients): W1 [H][n_in], b1 [H],
 * W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out] at the offsets sur_param_offsets reports
 * (each tensor starts on a 16-byte boundary; y = x W^T + b).
 */
#ifndef SUR_H
#define SUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SUR_OK 0
#define SUR_ERR_INVALID_ARG (-1)
#define SUR_ERR_ALLOC (-2)
#define SUR_ERR_CUDA (-3)

typedef struct sur_ctx sur_ctx;

/* Network n_in -> n_hidden -> n_hidden -> n_out with weights drawn uniformly in
 * +-1/sqrt(fan_in) from `seed`; max_batch = most rows one forward or training step handles. */
int sur_create(int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch, uint64_t seed,
               void *stream, sur_ctx **out);

int64_t sur_param_count(const sur_ctx *c);
int sur_param_offsets(const sur_ctx *c, int64_t *offsets6);
/* Replace the parameters (host FP32, sur_param_count values); resets the Adam state.    */
int sur_set_params(sur_ctx *c, const float *host);
int sur_get_params(sur_ctx *c, float *host);

/* y_dev [B][n_out] = network(x_dev [B][n_in]), any B >= 0 (processed in max_batch rows). */
int sur_forward(sur_ctx *c, const float *x_dev, int64_t B, float *y_dev);

/* Mean squared error of one batch (1 <= B <= max_batch) and its gradient with respect to
 * every parameter (host, sur_param_count values; either output may be NULL).             */
int sur_loss_grad(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float *loss_host,
                  float *grad_host);

/* Mean squared error over B >= 1 rows (host result).                                     */
int sur_loss(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float *loss_host);

/* One Adam step on one batch (1 <= B <= max_batch) with learning rate lr.               */
int sur_adam_step(sur_ctx *c, const float *x_dev, const float *t_dev, int64_t B, float lr);

/* `epochs` passes over n rows (X_dev [n][n_in], T_dev [n][n_out]) in shuffled mini-batches
 * of `batch` rows (a seeded permutation per epoch; the last n % batch rows of each
 * permutation are skipped). loss_host (may be NULL): mean mini-batch loss per epoch.
 * One epoch is captured in a CUDA graph on first use and replayed.                       */
int sur_train(sur_ctx *c, const float *X_dev, const float *T_dev, int64_t n, int32_t batch,
              int32_t epochs, float lr, uint64_t seed, float *loss_host);

/* Proper orthogonal decomposition of solver snapshots (the basis whose coefficients the
 * network predicts): X_dev [n][D] binary32 snapshots (device), 2 <= n <= 32768,
 * 1 <= r <= min(48, n - 1). Writes mean_dev [D] (column means), phi_dev [D][r] (the r
 * leading orthonormal modes of the centred snapshots X_c), coef_dev [n][r] (X_c phi) and,
 * if not NULL, lam_host [r] (eigenvalues of X_c X_c^T, descending), frac_host (their share
 * of the trace) and iters_host (subspace iterations taken). Each mode's sign makes its
 * largest-magnitude coefficient positive. Method of snapshots: the Gram matrix X_c X_c^T
 * (n x n binary64 on the device; binary32 products summed 32 at a time, accumulated in
 * binary64), its leading eigenvectors by subspace iteration with Rayleigh-Ritz in binary64
 * (block of min(n - 1, r + 16) vectors, until every residual is below 1e-11 of the top
 * eigenvalue, at most 1000 iterations), phi = X_c^T V / sqrt(lambda) in binary64.
 * Allocates its work space (n^2 + 3 n (r + 16) + D doubles) with cudaMalloc; runs on
 * stream and synchronises it.                                                           */
int sur_pod(const float *X_dev, int64_t n, int64_t D, int32_t r, float *mean_dev, float *phi_dev,
            float *coef_dev, double *lam_host, double *frac_host, int32_t *iters_host, void *stream);

/* Trust region of the trained network, so that the plain solver stays the fallback for
 * realisations the network was not trained on (the surrogate's inputs are KL
 * coefficients drawn from N(0, I)). The radius is the smallest Euclidean norm with at
 * least q n of the n training inputs X_dev [n][n_in] at or below it (0 < q <= 1; q = 1
 * gives the largest training norm); norms in binary64 on the device. radius_out (may be
 * NULL) receives it. Synchronises the stream.                                           */
int sur_fit_trust(sur_ctx *c, const float *X_dev, int64_t n, double q, double *radius_out);

/* flags_dev [B] (device int32): 1 where the input row x_dev [B][n_in] has a norm within
 * the trust radius, 0 where its prediction should be replaced by a solver run.
 * SUR_ERR_INVALID_ARG before sur_fit_trust. Asynchronous on the stream.                */
int sur_trust(sur_ctx *c, const float *x_dev, int64_t B, int32_t *flags_dev);

/* POD reconstruction u_dev [B][D] = mean_dev [D] + coef_dev [B][r] phi_dev [D][r]^T.     */
int sur_reconstruct(const float *coef_dev, const float *mean_dev, const float *phi_dev, int32_t B,
                    int64_t D, int32_t r, float *u_dev, void *stream);

/* Statistics of the fields u = mean + phi c implied by M predicted coefficient rows
 * coef_dev [M][r] (1 <= r <= 64): out_mean [D] = mean + phi mu_c and out_std [D] =
 * sqrt(diag(phi C_c phi^T)) with mu_c, C_c the coefficients' sample mean and covariance
 * (divisor M - 1). work_dev: device scratch of r + r * r floats.                        */
int sur_field_stats(const float *coef_dev, int32_t M, int32_t r, const float *mean_dev,
                    const float *phi_dev, int64_t D, float *work_dev, float *out_mean_dev,
                    float *out_std_dev, void *stream);

/* General product on the tensor cores (BF16 inputs, FP32 accumulation):
 * C[m][n] (row stride ldc) = sum_k A[m sam + k sak] B[k sbk + n sbn]; used for POD
 * projections, coefficients = (u - mean) phi.                                            */
int sur_matmul(const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk, int64_t sbn,
               float *C, int32_t M, int32_t N, int32_t K, int32_t ldc, void *stream);

const char *sur_last_error(const sur_ctx *c);
void sur_destroy(sur_ctx *c);

#ifdef __cplusplus
}
#endif

#endif /* SUR_H */
