/*
 * lt_nn.h - C ABI of the learned warm start's layers (no counterpart in the
 * paper; a 3D U-Net that maps a normalised back-projection A^T y to an initial
 * volume for the reconstruction of Sec. V).
 *
 * Tensors are channels-last: [batch][D][H][W][C], C fastest.  Activations and
 * weights are bfloat16 (uint16_t bit patterns), accumulation is float32.
 * Convolution weights are [Co][27][Ci] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)),
 * 3x3x3 with zero padding 1, stride 1.  Channel counts must be multiples of
 * 16 (pad the network input to 16 channels).  All pointers are device
 * pointers owned by the caller; calls are asynchronous on the stream and
 * return LT_EINVAL for bad sizes, LT_ECUDA for launch errors.
 */
#ifndef LT_NN_H
#define LT_NN_H

#include <stdint.h>

#include "lt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out[v][o_off + co] = act(b[co] + sum_{tap,ci} w[co][tap][ci] in[v + tap][ci]);
 * act = ReLU if relu != 0.  out has o_stride channels per voxel (>= o_off+Co),
 * so decoder outputs can be written into a concatenation buffer.  Output is
 * bfloat16 (out_bf) and/or float32 (out_f); either may be NULL. */
LT_API lt_status lt_nn_conv3d(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf,
                              float* out_f, int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                              int32_t Co, int32_t o_stride, int32_t o_off, int32_t relu, void* stream);

/* lt_nn_conv3d with an explicit kernel: LT_CONV_AUTO takes a tcgen05 kernel
 * wherever one applies and the warp-level MMA kernel elsewhere, LT_CONV_WARP_MMA
 * is the warp-level MMA kernel (every shape), LT_CONV_TCGEN05 the faster of
 * the two tcgen05 kernels (operands in shared memory, accumulators in tensor
 * memory), LT_CONV_TCGEN05_CHUNKED and LT_CONV_TCGEN05_ZWALK one of them.
 * Both need W a multiple of 64 and 16-byte aligned in, w and out_bf; the
 * chunked kernel (CTA = 2 x 2 output rows, input channels in chunks of 16)
 * needs H and D even, the z-walking kernel (CTA = 4 output rows walking 8
 * slices, a ring of input planes) Ci == 16, H a multiple of 4 and Co not a
 * multiple of 48.  Other shapes give LT_EUNSUPPORTED on those paths. */
enum {
  LT_CONV_AUTO = 0,
  LT_CONV_WARP_MMA = 1,
  LT_CONV_TCGEN05 = 2,
  LT_CONV_TCGEN05_CHUNKED = 3,
  LT_CONV_TCGEN05_ZWALK = 4
};
LT_API lt_status lt_nn_conv3d_ex(const uint16_t* in, const uint16_t* w, const float* b, uint16_t* out_bf,
                                 float* out_f, int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                                 int32_t Co, int32_t o_stride, int32_t o_off, int32_t relu, int32_t path,
                                 void* stream);

/* Synchronises the stream, then reports and clears the device status of the
 * tcgen05 kernels: LT_OK, or LT_ETIMEOUT if a bounded wait on the tensor core
 * gave up (that CTA's outputs were not written). */
LT_API lt_status lt_nn_device_status(void* stream);

/* Weight gradient: dw[co][tap][ci] += sum_v g[v][co] in[v + tap][ci] and
 * db[co] += sum_v g[v][co] (db may be NULL); float32 accumulation, g has Co
 * channels per voxel.  Deterministic: every CTA stores its partial sums in the
 * caller's device workspace `work` (work_floats floats, at least what
 * lt_nn_conv3d_wgrad_workspace reports for the same shape; contents on entry
 * do not matter, overwritten), and one kernel adds them to dw and db in a fixed
 * order, so repeated calls on the same inputs give the same bits.  LT_EINVAL
 * for channel counts not multiples of 16, NULL pointers or a short workspace;
 * `work` must not be shared with a call in flight on another stream. */
LT_API lt_status lt_nn_conv3d_wgrad(const uint16_t* in, const uint16_t* g, float* dw, float* db, float* work,
                                    int64_t work_floats, int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci,
                                    int32_t Co, void* stream);
/* Workspace (floats) lt_nn_conv3d_wgrad needs for this shape; a few MB to
 * tens of MB (one row of 27 Co Ci partial sums per CTA column). */
LT_API lt_status lt_nn_conv3d_wgrad_workspace(int32_t batch, int32_t D, int32_t H, int32_t W, int32_t Ci, int32_t Co,
                                              int64_t* floats);

/* wt[ci][tap][co] = w[co][26 - tap][ci]: the weights whose convolution is the
 * data gradient (the transposed convolution) of lt_nn_conv3d. */
LT_API lt_status lt_nn_conv3d_flip(const uint16_t* w, uint16_t* wt, int32_t Ci, int32_t Co, void* stream);

/* Elementwise helpers on n elements. */
LT_API lt_status lt_nn_f32_to_bf16(const float* x, uint16_t* y, int64_t n, void* stream);
LT_API lt_status lt_nn_bf16_to_f32(const uint16_t* x, float* y, int64_t n, void* stream);
/* g[i] = (y[i] > 0) ? g[i] : 0 (ReLU backward, in place on bfloat16). */
LT_API lt_status lt_nn_relu_backward(const uint16_t* y, uint16_t* g, int64_t n, void* stream);

/* 2x2x2 average pooling [b][D][H][W][C] -> [b][D/2][H/2][W/2][C] and its
 * adjoint (gradient); D, H, W even.  Channel strides/offsets as in conv. */
LT_API lt_status lt_nn_avgpool2(const uint16_t* in, uint16_t* out, int32_t batch, int32_t D, int32_t H, int32_t W,
                                int32_t C, int32_t i_stride, int32_t i_off, void* stream);
LT_API lt_status lt_nn_avgpool2_backward(const uint16_t* gout, uint16_t* gin, int32_t batch, int32_t D, int32_t H,
                                         int32_t W, int32_t C, int32_t i_stride, int32_t i_off, void* stream);
/* Nearest 2x upsampling of [b][d][h][w][C] into channels [o_off, o_off+C) of a
 * [b][2d][2h][2w][o_stride] tensor, and its adjoint (sum of the 8 children). */
LT_API lt_status lt_nn_upsample2(const uint16_t* in, uint16_t* out, int32_t batch, int32_t d, int32_t h, int32_t w,
                                 int32_t C, int32_t o_stride, int32_t o_off, void* stream);
LT_API lt_status lt_nn_upsample2_backward(const uint16_t* gout, uint16_t* gin, int32_t batch, int32_t d, int32_t h,
                                          int32_t w, int32_t C, int32_t o_stride, int32_t o_off, void* stream);
/* Copy channels [s_off, s_off+C) of a [v][s_stride] tensor into channels
 * [d_off, d_off+C) of a [v][d_stride] tensor (skip connections). */
LT_API lt_status lt_nn_copy_channels(const uint16_t* src, uint16_t* dst, int64_t voxels, int32_t C, int32_t s_stride,
                                     int32_t s_off, int32_t d_stride, int32_t d_off, void* stream);
/* Gradient norm and clipping factor of n float32 gradients g, on the device
 * and in a fixed order: out[0] = min(1, max_norm / ||g||) (1 when max_norm <=
 * 0; 0 when ||g|| is not finite), out[1] = ||g||.  work: device scratch of at
 * least LT_NN_NORM_WORK floats; out: 2 device floats.  Nothing is read back
 * to the host. */
#define LT_NN_NORM_WORK 256
LT_API lt_status lt_nn_grad_norm_clip(const float* g, int64_t n, float max_norm, float* work, float* out,
                                      void* stream);
/* Adam step on float32 master weights p (and their bfloat16 copy pb, may be
 * NULL) with gradient s g, s = *g_scale (a device float, e.g. out[0] of
 * lt_nn_grad_norm_clip; NULL means 1): m = b1 m + (1-b1) s g;
 * v = b2 v + (1-b2) (s g)^2; p -= lr mhat/(sqrt(vhat)+eps), mhat = m/(1-b1^step),
 * vhat = v/(1-b2^step). */
LT_API lt_status lt_nn_adam(float* p, uint16_t* pb, const float* g, const float* g_scale, float* m, float* v,
                            int64_t n, float lr, float b1, float b2, float eps, int32_t step, void* stream);

/* out[i] = a[i] + b[i] (bfloat16, float32 arithmetic). */
LT_API lt_status lt_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, int64_t n, void* stream);

/* Network input from a back-projection bp = A^T y and the majoriser diagonal
 * d: r[v] = bp[v] / d[v] (0 where d = 0) and *m = max_v r[v] (device float,
 * r >= 0), then u[v][0] = r[v] / *m, u[v][1..15] = 0 (bfloat16, 16 channels). */
LT_API lt_status lt_nn_prepare_input(const float* bp, const float* d, float* r, float* m, uint16_t* u, int64_t voxels,
                                     void* stream);
/* x0[v] = max(out[v][0], 0) * (*m): the warm start from the network output. */
LT_API lt_status lt_nn_unpack_output(const float* out, const float* m, float* x0, int64_t voxels, void* stream);
/* Mean-squared error of out[v][0] against target[v] / (*m): g[v][0] =
 * 2 (out - t) / V, g[v][1..15] = 0, *loss += sum (out - t)^2 / V. */
LT_API lt_status lt_nn_mse(const float* out, const float* target, const float* m, float* g, float* loss,
                           int64_t voxels, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LT_NN_H */
