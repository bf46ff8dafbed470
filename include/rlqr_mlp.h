/*
 * rlqr_mlp.h -- C ABI of the warm-start network of the nonlinear IPM: a
 * 3-layer perceptron with BF16 weights and activations (FP32 accumulation,
 * FP32 master weights, Adam), mapping an instance's (x0, goal) to an initial
 * primal trajectory for rlqr_ipm_init.  The paper has no learned component;
 * the network only proposes the starting point, and the IPM from that point
 * (or from the plain cold start) decides the result.
 *
 *   a0 = bf16(x_in)                      x_in [rows][n_in]  (n_in <= 16)
 *   h1 = bf16(relu(a0 W1^T + b1))        W1 [width][16]  (columns >= n_in are 0)
 *   h2 = bf16(relu(h1 W2^T + b2))        W2 [width][width]
 *   y  = h2 W3^T + b3                    W3 [n_out_pad][width], y FP32
 * with width a multiple of 16 (<= 1024) and n_out_pad = n_out rounded up to
 * 16.  Loss = mean over rows and the n_out real columns of (y - t)^2.
 * Backward: dy = bf16(2 (y - t) / (rows n_out)); dW3 = dy^T h2, db3 = sum dy;
 * dz2 = bf16((dy W3) * [h2 > 0]); dW2 = dz2^T h1, db2 = sum dz2;
 * dz1 = bf16((dz2 W2) * [h1 > 0]); dW1 = dz1^T a0, db1 = sum dz1 (every
 * product a BF16 x BF16 tensor-core product with FP32 accumulation).
 *
 * Parameters: one FP32 array (master copy) in the order W1, b1, W2, b2, W3,
 * b3 (rlqr_mlp_param_count values), a BF16 copy of the weights (raw uint16
 * bits, same order, biases included) refreshed by every update, and the Adam
 * moments (two FP32 arrays of the same length).  All pointers DEVICE; rows a
 * multiple of 16, at most max_rows; params_bf16 and grad 32-byte aligned,
 * the workspace 256-byte aligned (RLQR_ERR_ARG / RLQR_ERR_WORKSPACE
 * otherwise); the workspace holds activations and
 * gradients for max_rows rows.
 */
#ifndef RLQR_MLP_H_
#define RLQR_MLP_H_

#include "rlqr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_in;     /* 1..16 */
  int32_t width;    /* multiple of 16, 16..1024 */
  int32_t n_out;    /* >= 1 */
  int32_t max_rows; /* multiple of 16 */
} rlqr_mlp_dims;

size_t rlqr_mlp_param_count(const rlqr_mlp_dims *d);
size_t rlqr_mlp_workspace_bytes(const rlqr_mlp_dims *d);

/* bf16 copy of the FP32 master parameters (round to nearest even). */
rlqr_status rlqr_mlp_sync_bf16(const rlqr_mlp_dims *d, const float *params, uint16_t *params_bf16,
                               rlqr_stream_t stream);

/* y [rows][n_out] (FP32) = network(x [rows][n_in] FP32). */
rlqr_status rlqr_mlp_forward(const rlqr_mlp_dims *d, const uint16_t *params_bf16, const float *x,
                             int32_t rows, float *y, void *ws, size_t ws_bytes,
                             rlqr_stream_t stream);

/* Loss and gradient (FP32, parameter order) of the rows idx[0..rows) of the
 * data set (x [*][n_in], t [*][n_out]); loss and grad are device pointers
 * (loss: 1 value). */
rlqr_status rlqr_mlp_grad(const rlqr_mlp_dims *d, const uint16_t *params_bf16, const float *x,
                          const float *t, const int32_t *idx, int32_t rows, float *loss,
                          float *grad, void *ws, size_t ws_bytes, rlqr_stream_t stream);

/* One Adam step (bias-corrected, step >= 1) on the FP32 master parameters
 * from grad, then the BF16 copy. */
rlqr_status rlqr_mlp_adam(const rlqr_mlp_dims *d, float *params, uint16_t *params_bf16,
                          float *m, float *v, const float *grad, int32_t step, float lr,
                          float beta1, float beta2, float eps, rlqr_stream_t stream);

/* One training step (rlqr_mlp_grad, then rlqr_mlp_adam: the same kernels)
 * whose step-dependent inputs are read on the device, so that the call can
 * be captured once into a CUDA graph and replayed for consecutive steps.
 * With s = *counter (device int32: steps of the sequence done so far) the
 * batch is the rows indices idx_all[s rows .. s rows + rows) and the Adam
 * step takes lr = sched[3 s], the bias corrections c1 = sched[3 s + 1] =
 * 1 - beta1^t and c2 = sched[3 s + 2] = 1 - beta2^t (t its global step
 * number); the call then increments *counter on the device.  idx_all,
 * sched, counter and loss are device pointers; the caller sizes idx_all
 * and sched for every step it replays. */
rlqr_status rlqr_mlp_train_step(const rlqr_mlp_dims *d, float *params, uint16_t *params_bf16,
                                float *m, float *v, float *grad, const float *x, const float *t,
                                const int32_t *idx_all, int32_t rows, int32_t *counter,
                                const float *sched, float beta1, float beta2, float eps,
                                float *loss, void *ws, size_t ws_bytes, rlqr_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RLQR_MLP_H_ */
