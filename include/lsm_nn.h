/*
 * lsm_nn.h -- C ABI of the learned warm start (liblsm.so).
 *
 * The paper motivates its solver as a generator of training data for
 * machine-learning design loops (Abstract; Section 4) but trains no model.
 * This library adds one: a 4-level convolutional U-Net (32/64/128/256
 * channels, 3x3 convolutions with ReLU, 2x2 max pooling, nearest upsampling,
 * skip concatenation, 1x1 output head) that maps (phase map, current
 * non-affine displacement, strain increment) to the displacement the plain
 * damped relaxation adds after an affine load step. Its prediction only moves
 * the relaxation's starting point; the relaxation then runs to the same
 * force-residual tolerance, so for an increment in which no spring breaks the
 * answer does not depend on the network (to that tolerance) and a poor
 * prediction only costs steps. Breaks are tested at every step of the
 * relaxation, so in an increment where springs break the changed transient
 * can change which of them break.
 *
 * Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
 * cores (forward, data-gradient and weight-gradient convolutions:
 * tcgen05.mma with operands staged by TMA and the accumulator in tensor
 * memory), FP32 master weights and Adam moments.
 * All tensor arguments are DEVICE pointers owned by the caller:
 *   network input   bf16 [B][H][W][32], channels 0..6 used (see
 *                   lsm_unet_prepare_input), the rest zero;
 *   network output  fp32 [B][H][W][2];
 *   displacements   fp32 [S][2][H][W] (component-major per specimen).
 * Calls are ordered on the network's stream (create) or the given stream.
 */
#ifndef LSM_NN_H
#define LSM_NN_H

#include "lsm.h"
#include "lsm_batch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_unet lsm_unet;

/* Network for H x W images (multiples of 8) and up to max_batch images per
 * call; weights He-initialised from seed. stream: cudaStream_t or NULL. */
lsm_status lsm_unet_create(int32_t height, int32_t width, int32_t max_batch, uint64_t seed, void *stream,
                           lsm_unet **out);
void lsm_unet_destroy(lsm_unet *u);
const char *lsm_unet_last_error(const lsm_unet *u);

/* Number of FP32 parameters; copy them out / in (host arrays). set_params
 * also resets the Adam moments. */
lsm_status lsm_unet_param_count(lsm_unet *u, int64_t *n);
lsm_status lsm_unet_get_params(lsm_unet *u, float *host, int64_t n);
lsm_status lsm_unet_set_params(lsm_unet *u, const float *host, int64_t n);

/* Forward pass of batch images (stream ordered). */
lsm_status lsm_unet_forward(lsm_unet *u, const void *in, float *out, int32_t batch);

/* Mean squared error against target (fp32 [B][H][W][2]) and its gradient
 * w.r.t. every parameter (host array of param_count floats, may be NULL);
 * loss (host, may be NULL). Synchronises. */
lsm_status lsm_unet_gradients(lsm_unet *u, const void *in, const float *target, int32_t batch, float *loss,
                              float *grad);

/* One Adam step (beta 0.9 / 0.999) on the mean squared error; loss (host,
 * may be NULL: then the call does not synchronise). */
lsm_status lsm_unet_train_step(lsm_unet *u, const void *in, const float *target, int32_t batch, float lr,
                               float *loss);

/* Input of S specimens (u8 phase [S][H][W], fp32 displacement u [S][2][H][W],
 * fp32 current strains eps [S], all device): channel 0 phase - 1.5; 1, 2 the
 * non-affine displacement per unit strain, (u_x - eps (X - xc), u_y) /
 * (eps W a / 2) (0 while eps == 0); 3 deps / 1e-3; 4 eps / 0.1; 5, 6 the
 * position (X - xc) / (W a / 2), (Y - yc) / (H a / 2). */
lsm_status lsm_unet_prepare_input(const uint8_t *phase, const float *u, const float *eps, float deps, int32_t S,
                                  int32_t H, int32_t W, double a, void *in, void *stream);

/* Training target: (u_relaxed - u_loaded) / (deps W a / 2), fp32 [S][H][W][2]. */
lsm_status lsm_unet_prepare_target(const float *u_loaded, const float *u_relaxed, float deps, int32_t S, int32_t H,
                                   int32_t W, double a, float *target, void *stream);

/* Prediction (fp32 [S][H][W][2]) -> displacement increment fp32 [S][2][H][W]. */
lsm_status lsm_unet_prediction_to_displacement(const float *pred, float deps, int32_t S, int32_t H, int32_t W,
                                               double a, float *du, void *stream);

/* (The network sees 7 input channels; its first convolution keeps 32 input
 * channels so that every convolution has a multiple of 32.) */

/* The implicit-GEMM convolution kernels on their own (tests):
 * out[b,y,x,out_c0+n] = act(bias[n] + sum_{tap,ci} in[b,y+dy,x+dx,in_c0+ci] W[n][tap][ci])
 * (taps 9: 3x3 with zero padding; taps 1: 1x1), NHWC bf16 with channel
 * strides in_cs/out_cs; Cin, Cout multiples of 32; relu 0/1. Channel
 * strides and offsets are multiples of 8 and bias (fp32, device, may be
 * NULL) is 16-byte aligned, else LSM_EINVAL; the output tile is staged in
 * shared memory and written by TMA stores. */
lsm_status lsm_nn_conv_forward(const void *in, int32_t in_cs, int32_t in_c0, int32_t Cin, const void *W,
                               const float *bias, void *out, int32_t out_cs, int32_t out_c0, int32_t Cout, int32_t B,
                               int32_t H, int32_t Wd, int32_t taps, int32_t relu, void *stream);

/* Fault injection and diagnostics: the number of polls after which a bounded
 * mbarrier wait of the tensor-core convolution's pipeline gives up (0: at
 * once; < 0 restores the default, 2^20, about a second at most). A
 * convolution that gives up waits for the copies and MMAs it has issued
 * (bounded by the default limit), frees its tensor memory, leaves its output
 * incomplete and makes the call that launched it return LSM_ETIMEOUT once;
 * the next call runs normally. Tests set 0 to exercise that path without a
 * GPU fault. Applies to later launches (stream-ordered on `stream`, then
 * synchronised). */
lsm_status lsm_nn_set_wait_limit(int32_t polls, void *stream);

/* dW[n][tap][ci] = sum_p grad[p][n] in[p shifted by tap][ci], db[n] = sum_p
 * grad[p][n] (db may be NULL); grad dense NHWC bf16 [B][H][W][Cout];
 * scratch: device fp32 workspace of scratch_floats (>= Cout * taps * Cin). */
lsm_status lsm_nn_conv_wgrad(const void *grad, int32_t Cout, const void *in, int32_t in_cs, int32_t in_c0, int32_t Cin,
                             int32_t B, int32_t H, int32_t Wd, int32_t taps, float *dW, float *db, float *scratch,
                             int64_t scratch_floats, void *stream);

/* Bridges between a batch of equal-size specimens and the network buffers:
 * displacement u = x - X of every specimen (fp32 [S][2][H][W]) and phases
 * (u8 [S][H][W], may be NULL); and adding a displacement increment to the
 * free components of every specimen (then re-evaluating accelerations,
 * Eq. 4). All specimens of the batch must be H x W. */
lsm_status lsm_batch_fields(lsm_batch *b, float *u, uint8_t *phase, int32_t H, int32_t W);
lsm_status lsm_batch_add_displacements(lsm_batch *b, const float *du, int32_t H, int32_t W);

#ifdef __cplusplus
}
#endif

#endif /* LSM_NN_H */
