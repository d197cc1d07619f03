/*
 * fdtd_mlp.h -- C ABI of the surrogate-network kernels (sm_103a).
 *
 * The paper has no learned component; this boundary serves the surrogate
 * that maps grounding-electrode parameters to transient impedance
 * waveforms produced by the FDTD path (an addition of this library).  It is
 * a plain multilayer perceptron: layers y = act(x W^T + b) with BF16
 * operands and FP32 accumulation on the tensor cores, GELU in its erf form,
 * mean-squared-error loss and Adam.
 *
 * Conventions for every call:
 *   - All array arguments are device pointers; row-major, rows = samples.
 *   - Weights of a layer with k inputs and n outputs are wt [n x k] (BF16,
 *     one output per row); bias [n] FP32.
 *   - Work is queued on cuda_stream (a cudaStream_t, NULL = legacy default);
 *     nothing synchronises.  Nothing is allocated.
 *   - Return value 0, FDTD_EINVAL (-1) for bad sizes / null required
 *     pointers, FDTD_ECUDA (-4) for a launch error.
 *   - Forward layers with k <= 256 run on the tcgen05 tensor cores (TMEM
 *     accumulator); their one wait (for the MMA chain) is bounded: when it
 *     runs out the layer skips its outputs and records the failure, which
 *     fdtd_mlp_check() reports.
 */
#ifndef FDTD_GB300_MLP_H
#define FDTD_GB300_MLP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { FDTD_ACT_NONE = 0, FDTD_ACT_GELU = 1 };

/* y = act(z), z = x wt^T + bias.  x: rows x k, BF16 (x_is_bf16 = 1) or FP32
 * (rounded to BF16 on load).  Outputs, each optional (NULL): y_bf16 and
 * y_f32 (rows x n), z_f32 (rows x n, the pre-activation the backward pass
 * needs). */
int fdtd_mlp_forward(const void *x, int x_is_bf16, int rows, int k, const void *wt, const float *bias, int n,
                     int act, void *y_bf16, float *y_f32, float *z_f32, void *cuda_stream);

/* Backward of one layer.  dy = dL/dy (rows x n, FP32); z the layer's
 * pre-activation (needed for GELU; may be NULL for FDTD_ACT_NONE).
 * dz_scratch (rows x n FP32, caller memory) receives dz = dy * act'(z).
 * Outputs, each optional: dw = dz^T x (n x k, FP32), db = column sums of dz
 * (n), dx = dz wt (rows x k, FP32).  dz and x enter the tensor cores as
 * BF16. */
int fdtd_mlp_backward(const void *x, int x_is_bf16, const float *z, const float *dy, int rows, int k, int n,
                      int act, const void *wt, float *dz_scratch, float *dw, float *db, float *dx,
                      void *cuda_stream);

/* Adam step on count FP32 parameters w with moments m, v and gradient g
 * (step t >= 1): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps) + lr wd w.
 * w_bf16 (optional) receives the updated weights rounded to BF16. */
int fdtd_mlp_adam(float *w, float *m, float *v, const float *g, void *w_bf16, int count, float lr, float beta1,
                  float beta2, float eps, float weight_decay, int t, void *cuda_stream);

/* Weighted squared error over rows x cols (row-major): loss[0] += scale *
 * sum_r w_r sum_c (y - target)^2 (atomic; clear it first) and
 * dy = 2 scale w_r (y - target).  row_weight [rows] may be NULL (w_r = 1);
 * with w_r = 1 / ||target_r||^2 the loss is the sum of squared relative L2
 * errors of the rows.  dy and loss are each optional. */
int fdtd_mlp_mse(const float *y, const float *target, const float *row_weight, int rows, int cols, float scale,
                 float *dy, float *loss, void *cuda_stream);

/* err[r] = ||y_r - target_r|| / ||target_r|| (the plain norm of the
 * difference when target_r is zero), rows x cols row-major. */
int fdtd_mlp_row_rel_err(const float *y, const float *target, int rows, int cols, float *err, void *cuda_stream);

/* dst[r, :] = src[idx[r], :] for r < rows (FP32 rows of cols entries; idx
 * int32, each in range of src -- not checked). */
int fdtd_mlp_gather_rows(const float *src, const int *idx, int rows, int cols, float *dst, void *cuda_stream);

/* y[r, :] *= scale[r] in place. */
int fdtd_mlp_scale_rows(float *y, const float *scale, int rows, int cols, void *cuda_stream);

/* Synchronise cuda_stream and report whether a bounded wait inside a
 * network kernel ran out since the last call: FDTD_OK, FDTD_ETIMEOUT (-6,
 * the flag is then cleared) or FDTD_ECUDA. */
int fdtd_mlp_check(void *cuda_stream);

/* A whole network in one launch (inference).  Layers l = 0 .. n_layers-1
 * map sizes[l] inputs to sizes[l+1] outputs, y = act_l(x wt_l^T + bias_l);
 * the last layer's output is multiplied by out_scale and stored as FP32.
 * Limits: 1 <= n_layers <= 6, every layer input sizes[0 .. n_layers-1] <=
 * 256, and the weights must fit the kernel's shared memory (each CTA of a
 * four-CTA cluster holds a quarter of every layer's rows: about 130 KB for
 * 6 -> 256 -> 256 -> 256 -> 512); otherwise FDTD_EINVAL.
 * The weights enter as a packed image (device memory, 16-byte aligned,
 * fdtd_mlp_net_pack_bytes bytes, written by fdtd_mlp_net_pack from the
 * BF16 wt_l [sizes[l+1] x sizes[l]]; re-pack after the weights change).
 * x: rows x sizes[0] FP32 (rounded to BF16 on load); y: rows x
 * sizes[n_layers] FP32; acts: host array of n_layers activation codes;
 * bias: host array of n_layers device pointers (NULL array or entry = no
 * bias).  Each output equals, bit for bit, the chain of fdtd_mlp_forward
 * layers (BF16 hidden activations) followed by the scaling.  Its waits are
 * bounded as in fdtd_mlp_forward (fdtd_mlp_check reports a timeout). */
int fdtd_mlp_net_pack_bytes(const int *sizes, int n_layers, size_t *bytes);
int fdtd_mlp_net_pack(const int *sizes, int n_layers, const void *const *wt, void *image, void *cuda_stream);
int fdtd_mlp_net_forward(const float *x, int rows, const int *sizes, int n_layers, const int *acts,
                         const void *image, const float *const *bias, float out_scale, float *y, void *cuda_stream);

/* FP32 -> BF16 conversion (round to nearest even) of count elements. */
int fdtd_mlp_to_bf16(const float *src, void *dst, int count, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FDTD_GB300_MLP_H */
