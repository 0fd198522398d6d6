/* Kernels of the learned warm start: a small convolutional encoder-decoder
 * that maps a cavity's obstacle mask, Rayleigh and Prandtl numbers to an
 * initial (u/U0, v/U0, T) for the LBM-FVM iteration, trained on steady fields
 * that the batched solver generates.  The paper has no such network; the
 * iteration started from the predicted state runs to the same residual as
 * from rest, so it is both the fallback and the measure of the prediction's error.
 *
 * Conventions (every entry point):
 * - BF16 tensors are passed as uint16_t pointers (IEEE bfloat16 bit
 *   patterns); activations are NHWC, element (b, y, x, c) at
 *   ((b * H + y) * W + x) * ld + c, where ld >= C is the tensor's channel
 *   stride, so that a tensor can be a channel slice of a wider one (the
 *   decoder's concatenation buffers).  Pointers point at channel 0 of the
 *   slice.
 * - 3x3 convolutions are cross-correlations with zero padding 1; weights are
 *   [Cout][9][Cin] with tap k = 3 ky + kx reading input (y + ky - 1,
 *   x + kx - 1).  Products are BF16 x BF16 on the tensor cores (tcgen05.mma,
 *   FP32 accumulation in tensor memory) for the forward and adjoint
 *   convolutions, warp-level mma for the weight gradient.
 * - The activation is the leaky ReLU with slope 1/16; its derivative is taken
 *   from the sign of the activation's output.
 * - All pointers are device pointers unless stated; stream is a cudaStream_t
 *   (NULL = legacy stream); every call only enqueues work.
 * - Return: 0 (LBMFVM_OK) or a negative status: -1 invalid argument (shape,
 *   alignment, NULL), -3 a CUDA error.  lbmfvm_sg_last_error() gives the
 *   message of the calling thread's last failure.
 * - Shape rules: H % 8 == 0 and 16 <= W with W % 16 == 0 for 3x3
 *   convolutions (W <= 240 for the forward and adjoint ones, whose padded
 *   rows of W + 8 positions form one TMA box row); Cin % 16 == 0 and
 *   Cout % 32 == 0, Cout <= 256 for the
 *   forward and adjoint convolutions; channel strides multiples of 8 and slice
 *   pointers 16-byte aligned.
 */
#ifndef LBMFVM_SURROGATE_H
#define LBMFVM_SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Modes of lbmfvm_sg_conv3x3's epilogue. */
#define LBMFVM_SG_LINEAR 0   /* y = conv(x) + bias */
#define LBMFVM_SG_LEAKY 1    /* y = leaky(conv(x) + bias) */
#define LBMFVM_SG_DLEAKY 2   /* y = conv(x) * leaky'(m): backward through the previous activation */

/* y (B x H x W x Cout, BF16) from x (B x H x W x Cin, BF16), weights w
 * ([Cout][9][Cin], BF16), bias (Cout floats, ignored by LBMFVM_SG_DLEAKY, may
 * be NULL) and, for LBMFVM_SG_DLEAKY, m (B x H x W x Cout, BF16, stride ldm):
 * the output of the activation whose input gradient y is. */
int lbmfvm_sg_conv3x3(const uint16_t *x, int32_t ldx, const uint16_t *w, const float *bias, uint16_t *y,
                      int32_t ldy, const uint16_t *m, int32_t ldm, int32_t B, int32_t H, int32_t W, int32_t Cin,
                      int32_t Cout, int32_t mode, void *stream);

/* Weights of the adjoint convolution: wt[ci][8 - k][co] = w[co][k][ci] (BF16),
 * so that lbmfvm_sg_conv3x3 with wt maps an output gradient (Cout channels)
 * to the input gradient (Cin channels). */
int lbmfvm_sg_flip(const uint16_t *w, uint16_t *wt, int32_t Cin, int32_t Cout, void *stream);

/* Accumulates the weight and bias gradients of a 3x3 convolution:
 * dw[co][k][ci] += sum_{b,y,x} dy[b,y,x,co] x[b, y+ky-1, x+kx-1, ci] and
 * db[co] += sum dy[.., co] (FP32 arrays, db may be NULL).  Accumulation order
 * varies from call to call (FP32 atomics). */
int lbmfvm_sg_conv3x3_wgrad(const uint16_t *x, int32_t ldx, const uint16_t *dy, int32_t lddy, float *dw, float *db,
                            int32_t B, int32_t H, int32_t W, int32_t Cin, int32_t Cout, void *stream);

/* 2x2 average pooling: y (B x H/2 x W/2 x C) from x (B x H x W x C). */
int lbmfvm_sg_pool2(const uint16_t *x, int32_t ldx, uint16_t *y, int32_t ldy, int32_t B, int32_t H, int32_t W,
                    int32_t C, void *stream);
/* Its adjoint plus a second gradient, through an activation:
 * dx = (pool2'(dy) + add) * leaky'(m), where add and m may be NULL (no term,
 * no factor); dx, add and m are B x H x W x C, dy is B x H/2 x W/2 x C. */
int lbmfvm_sg_pool2_backward(const uint16_t *dy, int32_t lddy, const uint16_t *add, int32_t ldadd, const uint16_t *m,
                             int32_t ldm, uint16_t *dx, int32_t lddx, int32_t B, int32_t H, int32_t W, int32_t C,
                             void *stream);
/* Nearest-neighbour 2x up-sampling: y (B x 2H x 2W x C) from x (B x H x W x C). */
int lbmfvm_sg_upsample2(const uint16_t *x, int32_t ldx, uint16_t *y, int32_t ldy, int32_t B, int32_t H, int32_t W,
                        int32_t C, void *stream);
/* Its adjoint through an activation: dx (B x H x W x C) = (sum of the 2x2
 * children of dy) * leaky'(m), m (B x H x W x C) may be NULL (no factor). */
int lbmfvm_sg_upsample2_backward(const uint16_t *dy, int32_t lddy, const uint16_t *m, int32_t ldm, uint16_t *dx,
                                 int32_t lddx, int32_t B, int32_t H, int32_t W, int32_t C, void *stream);

/* Output layer: y[p][o] = b[o] + sum_c w[o][c] x[p][c] over P pixels, FP32
 * weights and output (Cout <= 8, Cin <= 64). */
int lbmfvm_sg_conv1x1(const uint16_t *x, int32_t ldx, const float *w, const float *b, float *y, int64_t P,
                      int32_t Cin, int32_t Cout, void *stream);
/* Its backward: dx = (dy w) * leaky'(x) (BF16, stride lddx; x is the output
 * of the activation feeding the layer), dw += dy^T x, db += sum dy (FP32). */
int lbmfvm_sg_conv1x1_backward(const uint16_t *x, int32_t ldx, const float *w, const float *dy, uint16_t *dx,
                               int32_t lddx, float *dw, float *db, int64_t P, int32_t Cin, int32_t Cout, void *stream);

/* Masked mean squared error over P pixels with C channels: n = C * (number of
 * pixels with fluid != 0); *loss (device double) += sum over fluid pixels of
 * (pred - target)^2 / n; dpred = 2 (pred - target) / n at fluid pixels, 0
 * elsewhere.  n is passed by the caller (n_inv = 1 / n). */
int lbmfvm_sg_mse(const float *pred, const float *target, const uint8_t *fluid, int64_t P, int32_t C, double n_inv,
                  float *dpred, double *loss, void *stream);

/* One Adam update (Kingma and Ba, 2015) of n FP32 parameters p with
 * gradients g and moments m, v (step t >= 1); p_bf16 (may be NULL) receives
 * the updated parameters rounded to BF16. */
int lbmfvm_sg_adam(float *p, const float *g, float *m, float *v, uint16_t *p_bf16, int64_t n, float lr, float beta1,
                   float beta2, float eps, int32_t t, void *stream);

/* Network input: x (B x H x W x 16, BF16) with channel 0 the solid mask
 * (mask[b][y][x] != 0 -> 1), channels 1, 2 the per-sample scalars s[b][0],
 * s[b][1] (normalised log10 Ra and Pr) and channels 3..15 zero. */
int lbmfvm_sg_encode(const uint8_t *mask, const float *scalars, uint16_t *x, int32_t B, int32_t H, int32_t W,
                     void *stream);

/* Mask of an nx x ny cavity sampled at the cell centres of an H x W grid:
 * out[y][x] = mask[floor((y + 1/2) ny / H)][floor((x + 1/2) nx / W)]. */
int lbmfvm_sg_resample_mask(const uint8_t *mask, int32_t nx, int32_t ny, uint8_t *out, int32_t H, int32_t W,
                            void *stream);

/* Initial fields of an nx x ny cavity from a prediction pred (H x W x 3 FP32:
 * u/U0, v/U0, T): bilinear interpolation at node (i, j) from the point
 * ((i + 1/2) W / nx - 1/2, (j + 1/2) H / ny - 1/2) of the prediction grid
 * (clamped at its edges), u, v times U0, T clipped to [0, 1], zero velocity on
 * solid nodes (mask != 0, may be NULL) and on the box walls.  u, v, T: nx*ny
 * floats each, row-major. */
int lbmfvm_sg_resample_fields(const float *pred, int32_t H, int32_t W, const uint8_t *mask, int32_t nx, int32_t ny,
                              float U0, float *u, float *v, float *T, void *stream);

/* Synchronises stream and reads the status word of the 3x3 convolution's
 * bounded device waits: 0, or -4 if a wait ran out since the last check (that
 * launch's output was not written; the word is cleared), -3 on a CUDA error. */
int lbmfvm_sg_check(void *stream);

/* Fault-injection hook for testing the bounded waits of the forward and
 * adjoint convolutions: block 0 of the next lbmfvm_sg_conv3x3 launch skips its
 * first staged load, so that the waits for it give up after about a second
 * each; that block's output is not written, the status word is set (the next
 * lbmfvm_sg_check returns -4) and the block drains what it issued before it
 * returns.  Nothing faults and the CUDA context stays usable.  Returns 0. */
int lbmfvm_sg_inject_stall(void);

const char *lbmfvm_sg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBMFVM_SURROGATE_H */
