/*
 * lskum_mlp.h -- C ABI of the warm-start surrogate of the q-LSKUM solver.
 *
 * A coordinate/condition MLP predicts the flow field (rho, u1, u2, p) at
 * every point from (x, y, wall distance, Mach, alpha) so that a solve can
 * start from it instead of the uniform free stream; the solver (lskum.h)
 * then iterates to convergence, so the prediction only changes the starting
 * point, never the converged answer. The paper has no counterpart: it
 * starts every solve from the free stream (Algorithm 1, preprocessor()).
 *
 * Network: 21 input features (zero-padded to LSKUM_MLP_IN_PADDED) -> five
 * hidden layers of LSKUM_MLP_WIDTH (tanh) -> LSKUM_MLP_OUT linear outputs
 * (six linear layers). Training and inference run in hand-written CUDA
 * kernels: BF16 tensor-core GEMMs (mma.sync m16n8k16, or tcgen05 for the
 * forward pass of the 256-wide layers, see lskum_mlp_set_gemm) accumulating
 * in FP32, FP32 master weights, Adam.
 *
 * Parameters (flat FP32, host order): for l = 0..5: W_l [out_l x in_l]
 * row-major, then b_l [out_l]; in_0 = LSKUM_MLP_IN_PADDED (columns 21..31
 * of W_0 are forced to zero), out_5 = LSKUM_MLP_OUT.
 *
 * Pointers named *_dev are DEVICE pointers (the caller owns them); host
 * pointers are copied. Return codes are those of lskum.h; the detail of a
 * failure is in lskum_last_error(). Calls synchronise the handle's stream.
 */
#ifndef LSKUM_MLP_H
#define LSKUM_MLP_H

#include <stdint.h>

#include "lskum.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LSKUM_MLP_LAYERS 6
#define LSKUM_MLP_WIDTH 256
#define LSKUM_MLP_IN 21
#define LSKUM_MLP_IN_PADDED 32
#define LSKUM_MLP_OUT 4

typedef struct lskum_mlp lskum_mlp;

/* Total number of parameters (weights and biases). */
int64_t lskum_mlp_num_params(void);

/* Creates a network for batches of up to `capacity` samples (1..2^24).
 * proj: host 8 x 2 Fourier projection matrix (rows P_k; features sin/cos of
 * P_k . (x, y)). Parameters start at zero: call lskum_mlp_set_params. */
int lskum_mlp_create(int64_t capacity, const float* proj, lskum_mlp** out);
void lskum_mlp_destroy(lskum_mlp* h);

/* Host FP32 parameter vector in/out (n == lskum_mlp_num_params()). set also
 * resets the Adam moments and step count. */
int lskum_mlp_set_params(lskum_mlp* h, const float* params, int64_t n);
int lskum_mlp_get_params(lskum_mlp* h, float* params, int64_t n);

/* Feature encoding: raw_dev n x 5 (x, y, wall distance, M, alpha in
 * degrees) -> feat_dev n x LSKUM_MLP_IN_PADDED FP32:
 * [x/10, y/10, ln(d + 1e-3)/5, (M - 0.55) 4, (alpha - 1)/5,
 *  sin(P_k . (x, y)) k < 8, cos(P_k . (x, y)) k < 8, zeros]. */
int lskum_mlp_features(lskum_mlp* h, const float* raw_dev, int64_t n, float* feat_dev);

/* Inference: feat_dev n x 32 -> out_dev n x 4 (n <= capacity). */
int lskum_mlp_predict(lskum_mlp* h, const float* feat_dev, int64_t n, float* out_dev);

/* Forward + backward of the mean squared error against target_dev (n x 4)
 * without updating: gradients into host grads (may be NULL, length
 * num_params), loss into *loss (may be NULL). */
int lskum_mlp_gradients(lskum_mlp* h, const float* feat_dev, const float* target_dev, int64_t n,
                        float* grads, double* loss);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the batch;
 * *loss (may be NULL) receives the batch loss before the step. With loss
 * NULL the call returns once the work is queued on the handle's stream: the
 * caller keeps feat_dev and target_dev unchanged until that stream has run
 * it (lskum_mlp_sync, or order its own writes after it by running on the
 * same stream, see lskum_mlp_set_stream). With loss non-NULL it returns
 * after the step. */
int lskum_mlp_train_step(lskum_mlp* h, const float* feat_dev, const float* target_dev, int64_t n,
                         float lr, double* loss);

/* Waits for the handle's stream. */
int lskum_mlp_sync(lskum_mlp* h);

/* GEMM path of the forward pass's five 256-wide layers:
 *   LSKUM_MLP_GEMM_MMA_SYNC  warp-level mma.sync m16n8k16 (the default);
 *   LSKUM_MLP_GEMM_TCGEN05   fifth-generation tensor cores: one CTA per 128
 *     rows stages its X tile and W in shared memory, one thread issues
 *     tcgen05.mma (M 128, N 256, K 16) into a tensor-memory accumulator,
 *     the epilogue reads it back with tcgen05.ld (sm_100-family GPUs only).
 * Both accumulate BF16 products in FP32; results agree to the order of the
 * FP32 sums. The backward pass and the 4-wide output layer use mma.sync.
 * With tcgen05, a synchronising call returns LSKUM_ERR_TIMEOUT if a GEMM
 * gave up waiting for its accumulators (a bounded wait; the context stays
 * usable). Waits for the handle's stream first. Errors: INVALID_ARG
 * (unknown path). No counterpart in the paper. */
#define LSKUM_MLP_GEMM_MMA_SYNC 0
#define LSKUM_MLP_GEMM_TCGEN05 1
int lskum_mlp_set_gemm(lskum_mlp* h, int path);

/* Runs the handle's work on the caller's CUDA stream (a cudaStream_t; NULL
 * restores the handle's own stream). Work the caller queues on the same
 * stream -- refilling the batch buffers of lskum_mlp_train_step, say -- is
 * then ordered after the handle's. Waits for the previous stream first.
 * For the legacy default stream pass cudaStreamLegacy ((void*)0x1).
 * No counterpart in the paper (the warm start is not part of the method). */
int lskum_mlp_set_stream(lskum_mlp* h, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSKUM_MLP_H */
