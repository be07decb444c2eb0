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
 * Errors: GEA_ERR_INVAL (sizes, channel counts, mode, odd h or w with
 * UPADD, null x0 / wt / y, null x1 with UPADD), GEA_ERR_CUDA. */
int gea_conv3x3(int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout, int32_t mode,
                int32_t flags, const uint16_t *x0, const uint16_t *x1, const uint16_t *wt,
                const float *bias, void *y, int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GEA_NET_H */
