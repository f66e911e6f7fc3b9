/*
 * superscs_mlp.h -- C ABI of the learned warm start (libsuperscs.so).
 *
 * The paper has no counterpart: this is the warm-start extension of the
 * solver.  Any u0 is a valid start of Algorithm 1 (its convergence does not
 * depend on u0, Sec. 4.5), so a network that maps a problem's parameters to
 * an HSDE iterate close to the solution can only cost iterations, never
 * correctness; the solver's cold start stays the fallback.
 *
 * Network: y = W3 relu(W2 relu(W1 xn + b1) + b2) + b3 with xn = (x - in_mean)
 * / in_std and outputs in the units (y * out_std + out_mean).  GEMMs run on
 * the tensor cores in BF16 with FP32 accumulation; parameters, Adam state,
 * losses and normalisation are FP32.  Training minimises
 * 0.5 * mean over the batch and outputs of (y - tn)^2 with tn the normalised
 * target, by Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Matrices are row-major, one sample per row.  Every pointer argument of
 * the per-batch calls is a device pointer.  All calls are queued on the
 * stream given at creation; the ones that return a loss synchronise it.
 */
#ifndef SUPERSCS_MLP_H
#define SUPERSCS_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scs_mlp scs_mlp;

/* d_in -> d_hidden -> d_hidden -> d_out, batches of at most max_batch rows.
 * Weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a counter-based hash
 * of (seed, index); biases 0; normalisation identity.  Returns SCS_OK or a
 * negative code of superscs.h. */
int scs_mlp_create(int32_t d_in, int32_t d_hidden, int32_t d_out, int32_t max_batch, uint64_t seed,
                   void *cuda_stream, scs_mlp **out);

/* Per-column mean and standard deviation of X (rows x d_in) and Y (rows x
 * d_out), computed on the device and stored as the input / output
 * normalisation (a std below 1e-6 is replaced by 1). */
int scs_mlp_fit_normalization(scs_mlp *mlp, const float *X, const float *Y, int64_t rows);

/* One Adam step on a batch (B <= max_batch): forward, loss, backward,
 * update.  *loss (host) receives the batch loss before the update. */
int scs_mlp_train_step(scs_mlp *mlp, const float *X, const float *Y, int32_t B, float lr, float *loss);

/* Y (B x d_out, FP32, output units) = network(X). */
int scs_mlp_forward(scs_mlp *mlp, const float *X, int32_t B, float *Y);

/* Loss and gradients (in the parameter order W1, b1, W2, b2, W3, b3; W as
 * d_out_l x d_in_l row-major) of a batch without updating; grad (device,
 * scs_mlp_num_params floats) may be NULL; *loss is a host pointer. */
int scs_mlp_gradients(scs_mlp *mlp, const float *X, const float *Y, int32_t B, float *grad, float *loss);

int64_t scs_mlp_num_params(const scs_mlp *mlp);
/* Copy all parameters (same order as the gradients) to or from params
 * (host or device, FP32) -- checkpoint and restore. */
int scs_mlp_get_params(scs_mlp *mlp, float *params);
int scs_mlp_set_params(scs_mlp *mlp, const float *params);

void scs_mlp_destroy(scs_mlp *mlp);

#ifdef __cplusplus
}
#endif
#endif /* SUPERSCS_MLP_H */
