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

/* Internal buffers of a network, read back for checking each kernel on its
 * own inputs (the paper has no counterpart).  Activations and their
 * gradients are those of the last batch that ran forward (scs_mlp_forward,
 * scs_mlp_gradients or scs_mlp_train_step), B rows; the weight copies are the
 * BF16 operands the GEMMs read.  Buffers (element type, rows x cols):
 *   PARAMS, GRAD, ADAM_M, ADAM_V   FP32, 1 x num_params (order of the gradients;
 *                                  GRAD: the last gradients computed)
 *   IN_MEAN, IN_STD                FP32, 1 x d_in;  OUT_MEAN, OUT_STD  FP32, 1 x d_out
 *   XN   BF16, B x d_in    normalised input        H1, H2  BF16, B x d_hidden (after ReLU)
 *   Y    FP32, B x d_out   output, normalised units
 *   DY   FP32, B x d_out   d loss / d y;           DY16    BF16 copy of DY
 *   DH2, DH1   FP32, B x d_hidden, gradient at the pre-activation of layer 2 / 1;
 *   DH2_16, DH1_16   their BF16 copies
 *   W1 (d_hidden x d_in), W2 (d_hidden x d_hidden), W3 (d_out x d_hidden)   BF16
 *   W2T (d_hidden x d_hidden), W3T (d_hidden x d_out)   BF16 transposed copies
 * *rows, *cols, *elem_bytes (host, each may be NULL) receive the shape and the
 * element size (4 FP32, 2 BF16 bits).  With out non-NULL (host or device),
 * rows x cols packed row-major elements are copied there; the stream is
 * synchronised.  SCS_EINVAL for an unknown buffer. */
#define SCS_MLP_READ_PARAMS 0
#define SCS_MLP_READ_GRAD 1
#define SCS_MLP_READ_ADAM_M 2
#define SCS_MLP_READ_ADAM_V 3
#define SCS_MLP_READ_IN_MEAN 4
#define SCS_MLP_READ_IN_STD 5
#define SCS_MLP_READ_OUT_MEAN 6
#define SCS_MLP_READ_OUT_STD 7
#define SCS_MLP_READ_XN 8
#define SCS_MLP_READ_H1 9
#define SCS_MLP_READ_H2 10
#define SCS_MLP_READ_Y 11
#define SCS_MLP_READ_DY 12
#define SCS_MLP_READ_DY16 13
#define SCS_MLP_READ_DH2 14
#define SCS_MLP_READ_DH2_16 15
#define SCS_MLP_READ_DH1 16
#define SCS_MLP_READ_DH1_16 17
#define SCS_MLP_READ_W1 18
#define SCS_MLP_READ_W2 19
#define SCS_MLP_READ_W3 20
#define SCS_MLP_READ_W2T 21
#define SCS_MLP_READ_W3T 22
int scs_mlp_read(scs_mlp *mlp, int32_t what, void *out, int64_t *rows, int64_t *cols, int32_t *elem_bytes);

/* GEMM kernels of the network.  SCS_MLP_GEMM_TCGEN05 (the default):
 * fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory),
 * 128 x 128 tiles fed by TMA from tensor maps (128-byte swizzle, a four-stage
 * ring, producer / MMA / epilogue warps), K split across CTAs with a
 * fixed-order reduction when the tiles alone would leave most SMs idle.
 * SCS_MLP_GEMM_MMA: warp-level BF16 MMA (m16n8k16) from shared memory.  Both
 * compute C = A B^T in FP32 from BF16 operands; their results differ only in
 * FP32 summation order, and each is deterministic. */
#define SCS_MLP_GEMM_MMA 0
#define SCS_MLP_GEMM_TCGEN05 1

/* Choose the GEMM kernel of a network (default SCS_MLP_GEMM_TCGEN05). */
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
