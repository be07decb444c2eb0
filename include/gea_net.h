/*
 * gea_net.h -- C ABI of the tensor-core convolution layers of the learned
 * pressure-correction network (GB300, sm_103a).
 *
 * The network is an extension beyond the paper: a small convolutional
 * multigrid-style U-Net that proposes the correction e of the pressure
 * equation A e = r (Section 3, eq. p_prime_sd) from its residual. Its 3x3
 * convolutions run on the fifth-generation tensor cores (tcgen05.mma, BF16
 * operands in shared memory, FP32 accumulators in tensor memory).
 *
 * Conventions
 *  - Activations are bfloat16 (raw 16-bit patterns, uint16_t) in N x H x W x C
 *    order (channels last, no padding); FP32 outputs likewise.
 *  - Weights of a 3x3 layer are bfloat16 [cout][3][3][cin].
 *  - All pointers are device pointers; calls are enqueued on `stream`
 *    (a cudaStream_t; NULL for the legacy default stream) and do not wait.
 *  - Functions return 0 or a GEA_ERR_* code of gea.h.
 */
#ifndef GEA_NET_H
#define GEA_NET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Input forms of a convolution (fused into the layer's input load):
 *  PLAIN  xin = x0                          (x0: n x h x w x cin)
 *  POOL   xin = 2x2 average of x0           (x0: n x 2h x 2w x cin)
 *  UPADD  xin = x0 + nearest-neighbour prolongation of x1
 *                                           (x0: n x h x w x cin,
 *                                            x1: n x h/2 x w/2 x cin, h, w even)
 * The fused input is formed in FP32 from the bfloat16 operands and rounded
 * to bfloat16 (round to nearest even). */
enum { GEA_CONV_PLAIN = 0, GEA_CONV_POOL = 1, GEA_CONV_UPADD = 2 };

/* Output flags: RELU applies max(0, .) after the bias; OUT_F32 writes FP32
 * (otherwise bfloat16, rounded to nearest even). */
enum { GEA_CONV_RELU = 1, GEA_CONV_OUT_F32 = 2 };

/* 'same' 3x3 correlation with zero padding on the tensor cores:
 *   y[b,i,j,o] = bias[o] + sum_{di,dj,c} xin[b, i+di-1, j+dj-1, c] wt[o,di,dj,c]
 * (bias may be NULL: zero), accumulated in FP32. cin, cout in {16, 32, 64};
 * n, h, w >= 1. status (optional device int) receives GEA_ERR_TIMEOUT if a
 * wait for the tensor cores gave up (never expected); it is not cleared.
 * After such a give-up the CTA waits once more, again bounded, for its MMA
 * batch before it frees its tensor memory; if that wait also runs out, the
 * batch may still be writing, so after GEA_ERR_TIMEOUT treat the CUDA context
 * as lost (destroy it before further GPU work in the process).
 * Errors: GEA_ERR_INVAL (sizes, channel counts, mode, odd h or w with
 * UPADD, null x0 / wt / y, null x1 with UPADD), GEA_ERR_CUDA. */
int gea_conv3x3(int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout, int32_t mode,
                int32_t flags, const uint16_t *x0, const uint16_t *x1, const uint16_t *wt,
                const float *bias, void *y, int32_t *status, void *stream);

/* ---- the network ----
 *
 * Layers, in parameter order (k x k correlation with zero padding, weights
 * [cout][k][k][cin] then bias [cout], FP32 in the parameter vector):
 *   e0a 1->16, e0b 16->16                      level 0 (full size)
 *   e1a 16->32 (input: 2x2 average of e0b), e1b 32->32        level 1
 *   e2a 32->64 (input: average of e1b), e2b 64->64            level 2
 *   e3a 64->64 (input: average of e2b), e3b 64->64            level 3
 *   d2a 64->64 (input: e2b + prolonged e3b), d2b 64->32       level 2
 *   d1a 32->32 (input: e1b + prolonged d2b), d1b 32->16       level 1
 *   d0a 16->16 (input: e0b + prolonged d1b), d0b 16->16       level 0
 *   out 16->1, 1x1 kernel, no activation
 * (k = 3 except out). Every layer but out applies max(0, .) when the network
 * is created with GEA_NET_RELU, none otherwise (a linear network).
 *
 * Forward: per sample b, x = r_b / rms(r_b) (rms over the sample's h w
 * values; x = 0 if r_b = 0) rounded to bfloat16; the layers run on bfloat16
 * activations and weights with FP32 accumulation; the output y (FP32) is
 * the correction of the pressure equation for the residual r up to a
 * positive scale per sample (rms(r_b) / mean(c_b) when trained with
 * gea_net_energy). h, w multiples of 8.
 *
 * Training loss (gea_net_energy), per sample, with A the Helmholtz operator
 * (A e)_i = c_i e_i + sum_f a_f (e_i - e_N) given by c (h x w), ax
 * (h x (w+1), face j between columns j-1 and j, zero on the walls), az
 * ((h+1) x w), and A_hat = A / mean(c):
 *     L_b = (0.5 y_b . A_hat y_b - y_b . x_b) / (h w),   L = mean_b L_b,
 * minimal at y_b = A_hat^-1 x_b. */
typedef struct gea_net gea_net;

enum { GEA_NET_RELU = 1 };
enum { GEA_NET_LAYERS = 15 };

/* Number of FP32 parameters of the network. */
int64_t gea_net_param_count(void);

/* Layer table: for each of the GEA_NET_LAYERS layers, 6 int32 values
 * {cin, cout, k, activation (1/0), input kind (0 network input, 1 previous
 * layer, 2 average of a finer layer, 3 sum of a skip layer and a prolonged
 * coarser layer), level}. desc holds 6 * GEA_NET_LAYERS values. */
int gea_net_layout(int32_t *desc);

/* Create a network for batches of at most n_max samples of at most
 * h_max x w_max values; allocates the parameters (zero), the Adam moments
 * and the activation and gradient buffers on the current device.
 * Errors: GEA_ERR_INVAL (sizes < 8 or not multiples of 8, flags),
 * GEA_ERR_NOMEM, GEA_ERR_CUDA. */
int gea_net_create(int32_t n_max, int32_t h_max, int32_t w_max, int32_t flags, gea_net **out);
int gea_net_set_stream(gea_net *net, void *stream);

/* Copy the parameter vector in or out (gea_net_param_count FP32 values,
 * host or device memory, mem = GEA_MEM_HOST / GEA_MEM_DEVICE of gea.h).
 * set_params also resets the Adam moments and step count. */
int gea_net_set_params(gea_net *net, const float *theta, int32_t mem);
int gea_net_get_params(gea_net *net, float *theta, int32_t mem);

/* y = N(r) for n samples of h x w (device arrays, dense, FP32). Keeps the
 * activations for gea_net_backward. */
int gea_net_forward(gea_net *net, int32_t n, int32_t h, int32_t w, const float *r, float *y);

/* Energy loss of the last forward pass (see above) for the operators of its
 * n samples (device arrays c: n x h x w, ax: n x h x (w+1), az: n x (h+1) x w)
 * and its gradient dL/dy into dy (device, n x h x w). *loss (host)
 * receives L; synchronises. */
int gea_net_energy(gea_net *net, const float *c, const float *ax, const float *az, float *dy,
                   float *loss);

/* Gradient of sum(dy * y) over the last forward pass with respect to the
 * parameters, into grad (device, gea_net_param_count values). The data
 * gradients run on the tensor cores with the activation gradient rounded to
 * bfloat16; the weight gradients are FP32 sums on the CUDA cores. */
int gea_net_backward(gea_net *net, const float *dy, float *grad);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step count kept by the
 * network) on the gradient grad (device) with learning rate lr. */
int gea_net_adam(gea_net *net, const float *grad, float lr);

/* forward + energy + backward + Adam on one batch; *loss as gea_net_energy. */
int gea_net_train_step(gea_net *net, int32_t n, int32_t h, int32_t w, const float *r,
                       const float *c, const float *ax, const float *az, float lr, float *loss);

void gea_net_destroy(gea_net *net);

#ifdef __cplusplus
}
#endif
#endif /* GEA_NET_H */
