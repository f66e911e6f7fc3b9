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
 * stream given at creation; the ones that return a loss synchronise it and
 * report (SCS_ECUDA) a tensor-core GEMM of an earlier call whose bounded
 * wait expired.
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

/* GEMM kernels of the network.  SCS_MLP_GEMM_MMA: warp-level BF16 MMA
 * (m16n8k16) from shared memory.  SCS_MLP_GEMM_TCGEN05: fifth-generation
 * tensor cores (tcgen05.mma, accumulator in tensor memory), 128 x 128 tiles.
 * Both compute C = A B^T in FP32 from BF16 operands; their results differ
 * only in FP32 summation order. */
#define SCS_MLP_GEMM_MMA 0
#define SCS_MLP_GEMM_TCGEN05 1

/* Choose the GEMM kernel of a network (default SCS_MLP_GEMM_MMA). */
int scs_mlp_set_gemm(scs_mlp *mlp, int32_t impl);

/* C (M x N, FP32, row stride ldc) = A (M x K, BF16, row stride lda) times
 * B (N x K, BF16, row stride ldb) transposed, by the chosen kernel; device
 * pointers, A and B 16-byte aligned (null allowed when K = 0: C = 0), lda and
 * ldb multiples of 8 and >= K.
 * Synchronises the stream.  For checking the kernels against a reference;
 * allocates a 4-byte flag on the device per call.  SCS_EINVAL on bad
 * arguments, SCS_ECUDA if a launch failed or a tensor-core wait timed out. */
int scs_mlp_gemm_nt(int32_t impl, int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *B,
                    int32_t ldb, float *C, int32_t ldc, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SUPERSCS_MLP_H */
