/*
 * yfmlp.h -- C ABI of the S-parameter surrogate in libyeefdtd.so.
 *
 * The paper characterises every line by a full FDTD solve (Sec. II-A).  The surrogate maps
 * six line descriptors to the 50-ohm S11 and S21 at 128 frequencies, is trained on S-matrices
 * that the batched FDTD solver produces (yeefdtd.h, yf_batch_*), and hands queries it cannot
 * vouch for back to that solver.  All arithmetic runs in this library's kernels:
 * BF16 tcgen05 tensor-core GEMMs with FP32 accumulation in tensor memory, FP32 master
 * weights and Adam, FP32 loss and ensemble gate.
 *
 * Network (per ensemble member):
 *   x (6 descriptors, mapped to [-1, 1] by the per-feature range given at creation)
 *   -> z_1 = x W_1^T + b_1, a_1 = gelu(z_1)            W_1: 512 x 6
 *   -> three more hidden layers of 512, gelu           W_2..W_4: 512 x 512
 *   -> y = a_4 W_5^T + b_5                             W_5: 512 x 512
 *   gelu(u) = 0.5 u (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3)))
 *   y = [Re S11 (128 freqs), Im S11, Re S21, Im S21].
 *   Loss: mean over batch x 512 of (y - t)^2.  Adam with bias correction.
 *   Weights and activations enter the tensor cores as BF16; accumulation, biases, master
 *   weights, optimiser state and outputs are FP32.
 *
 * Parameter vector (host doubles, the layout of yf_mlp_set_params / get_params / grads):
 *   for l = 1..5: W_l row-major [out][in], then b_l [out]; YF_MLP_PARAMS entries in all.
 *
 * Conventions as in yeefdtd.h: every call returns a yf_status, yf_last_error() explains a
 * failure, handles are owned by the library until yf_mlp_destroy, arrays marked with a
 * yf_mem argument may be host or device memory, all device work is ordered on the stream
 * given at creation (NULL: the library creates one).  Calls that return results to the
 * host synchronise that stream.
 */
#ifndef YFMLP_H
#define YFMLP_H

#include "yeefdtd.h"

#ifdef __cplusplus
extern "C" {
#endif

#define YF_MLP_IN 6
#define YF_MLP_WIDTH 512
#define YF_MLP_OUT 512
#define YF_MLP_LAYERS 5
#define YF_MLP_PARAMS 1054208L

typedef struct yf_mlp yf_mlp;

/* members: ensemble size 1..8.  train_batch: rows per training step, a positive multiple of
 * 128.  max_query: largest yf_mlp_query batch (>= 1).  in_lo/in_hi [6]: range of each raw
 * descriptor, mapped linearly to [-1, 1] inside the input kernel (in_hi > in_lo).
 * The weights start at zero: call yf_mlp_set_params for every member before training. */
yf_status yf_mlp_create(int members, int train_batch, int max_query, const double *in_lo,
                        const double *in_hi, void *stream, yf_mlp **out);
yf_status yf_mlp_destroy(yf_mlp *m);

/* Replace member's weights (host doubles, rounded to FP32 masters and BF16 copies) and
 * reset its Adam state and step count. */
yf_status yf_mlp_set_params(yf_mlp *m, int member, const double *params);
/* Member's FP32 master weights as doubles. */
yf_status yf_mlp_get_params(yf_mlp *m, int member, double *params);
/* Adam hyper-parameters for subsequent steps (defaults 1e-3, 0.9, 0.999, 1e-8). */
yf_status yf_mlp_set_adam(yf_mlp *m, double lr, double beta1, double beta2, double eps);

/* Forward and backward pass of one member on one training batch, without an update:
 * x [train_batch][6] raw descriptors, t [train_batch][512] targets (float32, `where`).
 * *loss (nullable) receives the batch loss; grads (nullable, host) receives dLoss/dparams in
 * the parameter layout.  Synchronous. */
yf_status yf_mlp_grads(yf_mlp *m, int member, const float *x, const float *t, yf_mem where,
                       double *loss, double *grads);

/* One Adam step of one member on one batch (as yf_mlp_grads, then the update).  Asynchronous
 * unless loss is non-NULL. */
yf_status yf_mlp_train_step(yf_mlp *m, int member, const float *x, const float *t,
                            yf_mem where, double *loss);

/* Many Adam steps of one member from device-resident data, replayed from one captured CUDA
 * graph of the whole step (batch gather, forward, loss, backward, Adam, BF16 publish):
 *   x [n][6], t [n][512] float32 DEVICE arrays (the training set);
 *   idx [steps * train_batch] int32 DEVICE: rows of step s are idx[s*B .. s*B + B - 1], each in
 *     [0, n) (an out-of-range row stops that step's gather and makes yf_mlp_sync report
 *     YF_E_INVALID);
 *   lr [steps] float32 DEVICE: the learning rate of each step.
 * Asynchronous; the arrays must stay valid until the work completes (yf_mlp_sync).  The graph
 * is kept and reused while the same pointers and n are passed again. */
yf_status yf_mlp_fit(yf_mlp *m, int member, const float *x, const float *t, int n,
                     const int32_t *idx, const float *lr, long steps);

/* Wait for the handle's queued work; report a device-side failure (YF_E_TIMEOUT for a wait
 * that gave up, YF_E_INVALID for an out-of-range training row); *loss (nullable) = the loss
 * of the last training batch. */
yf_status yf_mlp_sync(yf_mlp *m, double *loss);

/* Ensemble inference: x [n][6] raw descriptors (1 <= n <= max_query, `where`).
 * y [n][512] receives the ensemble mean; est [n] (nullable) the disagreement
 * max over members, S entries (S11, S21) and frequencies of |S_member - S_mean| (complex
 * magnitude).  Outputs live in `out_where` memory: device outputs are written in place by the
 * ensemble kernel (stream-ordered, no synchronisation); host outputs go through the handle's
 * device buffers and synchronise the stream. */
yf_status yf_mlp_query(yf_mlp *m, const float *x, int n, yf_mem where, float *y, float *est,
                       yf_mem out_where);

/* Gate: flags[i] = (scale * est[i] > threshold) for i < n; *nflagged (nullable) the count.
 * est and flags in `where` memory.  scale calibrates the disagreement to the error it
 * predicts (measured on held-out FDTD solves by the caller). */
yf_status yf_mlp_gate(yf_mlp *m, const float *est, int n, double scale, double threshold,
                      yf_mem where, int32_t *flags, int *nflagged);

/* Launch accounting of one yf_mlp_query: *launches (nullable) = kernels it launches, and
 * *gemm_flops (nullable) = algorithmic tensor-core FLOPs per query row over all members
 * (2 * (6*512 + 3*512*512 + 512*512) per member). */
yf_status yf_mlp_query_stats(yf_mlp *m, int *launches, double *gemm_flops);

#ifdef __cplusplus
}
#endif

#endif
