/* unet.h -- C ABI of the warm-start network (liblbgb.so).
 *
 * The paper's method (Eqs. 1, 2/4, 7, 24-25) relaxes a droplet or slab to a
 * steady state.  This network predicts that steady state (rho, T) from the
 * case's T/T_c, G and initial liquid mask, and the handoff below turns the
 * prediction into the method's initial state (f = f^eq(rho, 0),
 * g = c_v T f^eq(rho, 0) via lb_init_device / lb_batch_init), after which the
 * method itself relaxes the remaining error.  The paper has no counterpart of
 * the network; mass and energy of the handoff follow the conservation of
 * Eq. (13) and sum_i C_i = 0 (Eq. 25).
 *
 * Network: 4-level U-Net, base width C (32 for the reference net; a multiple
 * of 32).  Encoder level l (width C 2^l): two 3x3 circular convolutions +
 * ReLU, 2x2 average pool between levels; decoder: nearest 2x upsampling,
 * concatenation [upsampled, skip] along channels, two 3x3 convolutions +
 * ReLU; head: 1x1 convolution C -> 2, no activation.  The input and output
 * planes are pixel-major ([N][H][W][c]); the BF16 activations inside the net
 * are stored row by row in blocks of 8 channels (un_get_tensor returns them
 * as NHWC).
 * Arithmetic: BF16 weights and activations (round to nearest even), FP32
 * accumulation on the tensor cores, FP32 bias, head, loss, gradients of the
 * weights and Adam state (FP32 master weights).
 *
 * Parameters are one flat float32 vector, layer by layer in the order
 * e0a e0b e1a e1b e2a e2b e3a e3b d2a d2b d1a d1b d0a d0b head, each as
 * W[cout][k][k][cin_stored] followed by b[cout] (un_layer_info gives the
 * table).  The network input has 3 channels, stored padded to 32 (weights of
 * the padding channels stay 0 under Adam because their gradient is 0).
 *
 * Errors: lb_status codes of lb.h; the message is in lb_last_error().
 * Ownership: the net owns its device memory; caller arrays are only read or
 * written during the call (asynchronous calls: until the stream reaches them).
 */
#ifndef LBGB_UNET_H
#define LBGB_UNET_H

#include <stddef.h>
#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { UN_LEVELS = 4, UN_IN = 3, UN_IN_PAD = 32, UN_OUT = 2, UN_LAYERS = 15 };

typedef struct {
    int32_t H, W;       /* image size, multiples of 8 (three 2x2 pools)      */
    int32_t max_batch;  /* largest N any call may use                       */
    int32_t base;       /* base width C, a multiple of 32 (reference net: 32) */
} un_config;

typedef struct un_net un_net; /* opaque */

/* Number of parameters of the network cfg describes (-1 if cfg is invalid). */
int64_t un_param_count(const un_config* cfg);

/* Layer k (0..UN_LAYERS-1) of the flat parameter layout: stored input
 * channels, output channels, kernel size (3 or 1) and the offset of its W in
 * the flat vector (b follows W).  LB_ERR_ARG for k out of range. */
lb_status un_layer_info(const un_config* cfg, int32_t k, int32_t* cin, int32_t* cout,
                        int32_t* ksize, int64_t* offset);

/* Create a net on the device of `stream` (NULL: the current device and a
 * stream of its own, non-blocking).  Parameters start at zero; set them with
 * un_set_params.  LB_ERR_ARG for H, W not multiples of 8, base not a
 * multiple of 32 or max_batch < 1; LB_ERR_OOM if the activations do not fit.
 * Every asynchronous call below runs on that stream and reads its device
 * inputs there: the caller orders their production before the call and keeps
 * them alive and unchanged until the net's stream has passed it (an input
 * written on another stream, or freed to an allocator that hands its memory
 * to other streams' work, races with the net). */
lb_status un_create(const un_config* cfg, void* stream, un_net** out);

/* Copy all n = un_param_count parameters in (host or device float32; resets
 * the Adam moments and step count) or out (host float32).  Synchronise. */
lb_status un_set_params(un_net* net, const float* params, int64_t n);
lb_status un_get_params(un_net* net, float* params, int64_t n);

/* Gradient of the last un_loss_grad / un_train_step (host float32, n values). */
lb_status un_get_grads(un_net* net, float* grads, int64_t n);

/* Forward pass: d_in = device float32 [N][H][W][3] (normalised T/T_c, G and
 * mask planes), d_out = device float32 [N][H][W][2] (normalised rho, T).
 * 1 <= N <= max_batch.  Asynchronous. */
lb_status un_forward(un_net* net, int32_t N, const float* d_in, float* d_out);

/* Forward pass, mean squared error against d_target (device float32
 * [N][H][W][2]) and its gradient in every parameter (kept in the net).
 * *loss (may be NULL; then the call stays asynchronous) receives the loss;
 * with loss != NULL the call synchronises. */
lb_status un_loss_grad(un_net* net, int32_t N, const float* d_in, const float* d_target,
                       double* loss);

/* One Adam step (bias-corrected; step count kept in the net) on the FP32
 * master weights with the last gradient; refreshes the BF16 copies.
 * Asynchronous. */
lb_status un_adam_step(un_net* net, double lr, double beta1, double beta2, double eps);

/* un_loss_grad followed by un_adam_step. */
lb_status un_train_step(un_net* net, int32_t N, const float* d_in, const float* d_target,
                        double lr, double* loss);

/* Introspection for tests: copy an internal tensor of the last forward /
 * backward pass to host float32 (NHWC over the last call's N, its stored
 * channels; n must equal its size).  Forward tensors: UN_T_X0 (padded input,
 * 32 channels), UN_T_A + l (first encoder conv output of level l = 0..3),
 * UN_T_CAT + l (l = 0..2: [upsampled level l+1 output, skip_l]), UN_T_P + l
 * (pooled skip_l), UN_T_C + l (first decoder conv output of level l),
 * UN_T_D0 (head input).  Gradient tensors (UN_T_GRAD + id): the gradient of
 * the loss at the stored tensor for CAT and P, and at the pre-activation of
 * the producing convolution for A, C, D0, UP + l (l = 1..3: the convolution
 * whose output is upsampled into CAT + l - 1) and SKIP + l (l = 0..2: the
 * second encoder convolution of level l).  LB_ERR_ARG for an unknown id or a
 * wrong n.  Synchronises. */
enum {
    UN_T_X0 = 0,
    UN_T_A = 10,
    UN_T_CAT = 30,
    UN_T_P = 40,
    UN_T_C = 50,
    UN_T_D0 = 60,
    UN_T_UP = 70,
    UN_T_SKIP = 80,
    UN_T_GRAD = 100
};
lb_status un_get_tensor(un_net* net, int32_t id, float* host, int64_t n);

lb_status un_synchronize(un_net* net);

/* Release the net.  NULL is accepted. */
lb_status un_free(un_net* net);

/* Warm-start handoff for N cases of H x W sites (all pointers device).
 * The network outputs deviations from the case's initial fields; from the
 * prediction d_pred [N][H][W][2]:
 *   rho_hat = max(rho0 + rho_dev_scale y0, rho_floor),
 *   T_hat = T0 (1 + t_dev_scale y1)
 * (a zero prediction gives back the initial state).
 * Per case, with lo/hi the extreme values of rho_hat:
 *   1. rho1 = rho_hat + lam (rho_hat - lo)(hi - rho_hat): mass moved inside
 *      the interfaces only (the weight vanishes in both bulk phases), with
 *      lam = (sum rho0 - sum rho_hat) / sum of the weight, limited to
 *      |lam| (hi - lo) <= 1 so that rho1 stays within [lo, hi];
 *   2. rho = rho1 sum(rho0) / sum(rho1): exactly the initial mass (Eq. 13);
 *   3. T = T_hat sum(rho0 T0) / sum(rho T_hat): the initial energy (conserved
 *      under Eq. 24, sum_i C_i = 0).
 * d_rho0, d_T0: the case's initial fields (float64 [N][H][W]); d_rho, d_T:
 * float64 outputs of the same shape, ready for lb_init_device / lb_batch_init.
 * One block per case, sums in FP64 in a fixed order.  Asynchronous on
 * `stream`.  LB_ERR_ARG for NULL pointers or empty sizes. */
lb_status un_warm_fields(int32_t N, int32_t H, int32_t W, const float* d_pred, double rho_dev_scale,
                         double rho_floor, double t_dev_scale, const double* d_rho0,
                         const double* d_T0, double* d_rho, double* d_T, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBGB_UNET_H */
