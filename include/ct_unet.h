/*
 * ct_unet.h -- C ABI of the learned warm start: a U-Net with BF16 3x3
 * convolutions and FP32 accumulation on the tensor cores, trained on pairs
 * the relaxed OS-LALM solver generates (FBP image -> converged PWLS
 * solution x*) and used as the solver's initial image.  The paper has no
 * counterpart: Algorithm 1 starts from "an initial (FBP) image"; this module
 * supplies a better one and the plain FBP start remains the fallback.
 *
 * Conventions as in ct.h: device pointers to caller-owned memory, NULL
 * stream = legacy default stream, host-side validation with a status and
 * ct_last_error() message.  BF16 buffers are passed as void* (IEEE bfloat16
 * bit patterns, 16-byte aligned).
 */
#ifndef CT_UNET_H
#define CT_UNET_H

#include "ct.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Tensor-core GEMM C = A B^T: A [M][K], B [N][K] BF16 row-major (K
 * contiguous), C [M][N] FP32 row-major (overwritten).  K must be a positive
 * multiple of 8; A and B 16-byte aligned.  err: device int, set to 1 if a
 * bounded wait on the tensor-core pipeline gave up (then C is undefined).
 * Asynchronous on stream.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int *err, void *stream);

/* ------------------------------------------------------------------ single layers
 *
 * 3x3 convolution, padding 1, stride 1, BF16 NHWC tensors, FP32 accumulation
 * on the tensor cores.  The input is the channel concatenation of in1 (c1
 * channels; up1 != 0: stored at half resolution [B][H/2][W/2][c1] and read
 * through a nearest-neighbour 2x upsampling) and in2 ([B][H][W][c2], c2 may
 * be 0).  Weights w [co][3][3][c1+c2] BF16; bias [co] FP32.
 * c1 and co multiples of 16, c2 0 or a multiple of 8, pointers 16-byte
 * aligned.  err as for ct_gemm_bf16.  Asynchronous. */

/* out [B][H][W][co] = bf16(relu(conv(in) + bias)). */
ct_status ct_conv3x3_bf16(const void *in1, int c1, int up1, const void *in2, int c2, const void *w, const float *bias,
                          void *out, int B, int H, int W, int co, int *err, void *stream);

/* Gradient with respect to the input of a forward ct_conv3x3_bf16 whose
 * input was (m1, c1, up1, m2, c2): gout [B][H][W][co] is the gradient of its
 * pre-activation output; wt [c1+c2][3][3][co] is the flipped transpose of its
 * weights, wt[ci][8-t][co] = w[co][t][ci].  The result is multiplied by the
 * ReLU support of the input (m > 0) and split into g1 [B][H][W][c1] (full
 * resolution, also for an upsampled in1) and g2 [B][H][W][c2]. */
ct_status ct_conv3x3_bf16_dgrad(const void *gout, int co, const void *wt, const void *m1, int c1, int up1,
                                const void *m2, int c2, void *g1, void *g2, int B, int H, int W, int *err, void *stream);

/* FP32 floats of workspace ct_conv3x3_bf16_wgrad needs (split-K partial sums). */
long long ct_conv3x3_wgrad_workspace(int B, int H, int W, int ci, int co);

/* Weight and bias gradients of a 3x3 convolution: dw [co][3][3][c1+c2] and
 * db [co] (FP32, overwritten) = sums over pixels of gout x input patches. */
ct_status ct_conv3x3_bf16_wgrad(const void *in1, int c1, int up1, const void *in2, int c2, const void *gout, int co,
                                float *dw, float *db, float *work, long long work_floats, int B, int H, int W,
                                int *err, void *stream);

/* ------------------------------------------------------------------ U-Net
 *
 * Architecture (levels L, base channels C0, level l has C_l = C0 2^l
 * channels at resolution (H / 2^l, W / 2^l)):
 *   encoder level l: conv_a (3x3, C_{l-1} -> C_l; level 0: 1 -> C0), ReLU,
 *                    conv_b (3x3, C_l -> C_l), ReLU  (output s_l);
 *                    levels l > 0 take the 2x2 max-pool of s_{l-1};
 *   decoder level l (L-2 .. 0): conv_a over the channel concatenation of the
 *                    nearest-2x-upsampled deeper output (C_{l+1}) and s_l
 *                    (C_l) -> C_l, ReLU; conv_b (C_l -> C_l), ReLU (output f_l);
 *   output: y = x + (b_o + w_o . f_0) / in_scale (1x1 conv, residual).
 * The network sees x * in_scale.  Weights are BF16 in the convolutions
 * (FP32 master copies for the optimiser), activations and activation
 * gradients BF16 NHWC, accumulation FP32 (tensor memory).
 *
 * Parameter vector (FP32, the order of ct_unet_get_params): for each 3x3
 * layer in the order enc_0a, enc_0b, ..., enc_{L-1}a, enc_{L-1}b, dec_{L-2}a,
 * dec_{L-2}b, ..., dec_0a, dec_0b: W [C_out][3][3][C_in] then b [C_out]
 * (C_in of dec_la = C_{l+1} + C_l, upsampled part first); then w_o [C0], b_o. */
typedef struct ct_unet ct_unet; /* opaque; owns parameters, optimiser state and activation workspace */

typedef struct {
    int levels;         /* 2 .. 5 */
    int base_channels;  /* multiple of 16, at most 96 */
    int height, width;  /* multiples of 2^(levels-1) */
    int max_batch;      /* largest batch of forward/backward */
    float in_scale;     /* input multiplier (e.g. 1 / water attenuation) */
    unsigned long long seed; /* He-normal initialisation (SplitMix64 + Box-Muller on the host) */
} ct_unet_desc;

/* Create a network and its device workspace.  Errors: CT_EINVAL, CT_ENOMEM, CT_ECUDA. */
ct_status ct_unet_create(const ct_unet_desc *desc, ct_unet **out);
void ct_unet_destroy(ct_unet *net);
/* Number of FP32 parameters (-1 for NULL). */
long long ct_unet_num_params(const ct_unet *net);
/* Copy the parameters (which = 0) or the gradients of the last backward (which = 1) to a host array
 * of ct_unet_num_params floats.  Synchronous. */
ct_status ct_unet_get_params(const ct_unet *net, float *host, int which);
/* Replace the parameters from a host array (the layout above).  Synchronous. */
ct_status ct_unet_set_params(ct_unet *net, const float *host);
/* y = U-Net(x): x, y device [B][H][W] FP32, 1 <= B <= max_batch.  Keeps the activations for
 * ct_unet_backward.  Asynchronous on stream.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_unet_forward(ct_unet *net, const float *x, float *y, int B, void *stream);
/* Parameter gradients of sum(gy * y) for the last forward (same B): gy device [B][H][W].
 * Overwrites the gradient vector.  Asynchronous.  Errors: CT_EINVAL, CT_ECUDA. */
ct_status ct_unet_backward(ct_unet *net, const float *gy, int B, void *stream);
/* One Adam step (Kingma & Ba, with bias correction and decoupled weight decay) on the
 * parameters with the current gradients; refreshes the BF16 copies.  Asynchronous. */
ct_status ct_unet_adam(ct_unet *net, float lr, float beta1, float beta2, float eps, float weight_decay,
                       void *stream);
/* Synchronise the device and report whether a bounded tensor-core wait gave up since the last
 * call (CT_ETIMEOUT; results of the affected calls are undefined), else CT_OK. */
ct_status ct_unet_status(ct_unet *net);

#ifdef __cplusplus
}
#endif

#endif /* CT_UNET_H */
