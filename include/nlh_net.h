/*
 * nlh_net.h -- C ABI of the learned warm start and diagonal correction.
 *
 * The paper has no learned component (its solver is the deflated,
 * diagonally preconditioned CG of Sec. 4.3.2); this part adds one in front
 * of that solver and keeps the plain solver as the fallback, with the final
 * residual always checked by the FP64-accurate operator (nlh_solve's x0 and
 * diag_scale).
 *
 * The network, for B images of H x W pixels (H, W multiples of
 * 2^(levels-1)):
 *   - input planes per pixel [f, ln sigma, ln alpha] (f the noisy image);
 *   - a U-Net with `levels` resolutions and base << l channels at level l:
 *     two 3x3 convolutions (zero padding, bias, ReLU) per level, 2x2
 *     average pooling between encoder levels, nearest 2x upsampling and
 *     channel concatenation [upsampled, skip] on the way up, and a 1x1 head
 *     to two outputs (o0, o1) per pixel;
 *   - the initial guess u0 = mean(f) 1 + o0 (o0 = 0 is the deflated
 *     solver's own start (mean(b) / alpha) 1 for b = alpha f) and the
 *     preconditioner factor s = exp(clamp(o1, -4, 4)), so that
 *     P_c = P_a * s (P_a the Jacobi diagonal alpha + max(d - 1, 0),
 *     d = Gamma_full 1) is SPD by construction;
 *   - training loss per sample, with r0 = b - A u0 and e0 = u* - u0 taken
 *     from a snapshot of u0 (data, not differentiated):
 *       ||P_a (u0 - u*)||^2 / ||b - mean(b) 1||^2
 *         + beta ||r0 / (P_a s) - e0||^2 / ||e0||^2,
 *     averaged over the batch (the first term weighs the initial error the
 *     way the initial residual A (u* - u0) does for its rough part, relative
 *     to the residual of the solver's own start); Adam (Kingma & Ba 2015) on
 *     all parameters.
 *
 * Arithmetic: 3x3 weights and all activations are stored in bfloat16, every
 * product is accumulated in FP32 (tensor cores, mma m16n8k16), the head,
 * the loss and the parameter update run in FP32 / FP64, master parameters
 * are FP32.
 *
 * Parameter layout (nlh_net_set_params / get_params / get_grads: one flat
 * HOST float vector): for each layer in order, weights then bias; a 3x3
 * layer stores W[cout][3][3][cin], the head W[2][base]; layers are enc0a,
 * enc0b, enc1a, ..., enc{levels-1}b, dec{levels-2}a, dec{levels-2}b, ...,
 * dec0a, dec0b, head (nlh_net_layer gives each layer's sizes).
 *
 * Conventions as in nlh.h: device vectors are FP64 and owned by the caller;
 * `stream` is a cudaStream_t as void*; errors are nlh_status codes with a
 * message from nlh_last_error(); a network is not thread-safe.
 */
#ifndef NLH_NET_H
#define NLH_NET_H

#include "nlh.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nlh_net_s *nlh_net;

/* A batch of B images (B <= 64), all H x W.  f, ustar, e0, r0, deg are
 * DEVICE arrays of B*H*W doubles, image after image, row-major.  sigma and
 * alpha are HOST arrays of B values (> 0).  ustar, e0, r0, deg and beta are
 * read only by nlh_net_loss_grad (ustar and deg always, e0 and r0 when
 * beta > 0); deg is Gamma_full 1 of each image (nlh_plan_get_degrees). */
typedef struct {
    int B, H, W;
    const double *f;
    const double *sigma;
    const double *alpha;
    const double *ustar;
    const double *e0;
    const double *r0;
    const double *deg;
    double beta;
} nlh_net_batch;

/* Create a network with `levels` (2..4) resolutions and `base` (32 or 64)
 * channels at full resolution; parameters are zero until set.
 * Errors: NLH_ERR_ARG, NLH_ERR_OOM, NLH_ERR_CUDA. */
nlh_status nlh_net_create(int base, int levels, nlh_net *out);

/* Number of layers and of parameters (floats). */
nlh_status nlh_net_info(nlh_net net, int *n_layers, int64_t *n_params);

/* Sizes of layer i: input channels, output channels, kernel size (3 or 1). */
nlh_status nlh_net_layer(nlh_net net, int i, int *cin, int *cout, int *k);

/* Copy all parameters in (resets the Adam moments and step count) or out.
 * `count` must equal the parameter count.  Synchronous. */
nlh_status nlh_net_set_params(nlh_net net, const float *theta, int64_t count);
nlh_status nlh_net_get_params(nlh_net net, float *theta, int64_t count);

/* Copy out the gradient of the last nlh_net_loss_grad.  Synchronous. */
nlh_status nlh_net_get_grads(nlh_net net, float *grad, int64_t count);

/* Inference: u0 = mean(f) + o0 and scale = exp(clamp(o1, -4, 4)), DEVICE arrays
 * of B*H*W doubles (either may be NULL).  Stream-ordered, no sync. */
nlh_status nlh_net_forward(nlh_net net, const nlh_net_batch *batch, double *u0,
                           double *scale, void *stream);

/* Snapshot for the preconditioner term: e0 = ustar - u0 with u0 from the
 * current parameters (DEVICE, B*H*W).  Stream-ordered. */
nlh_status nlh_net_residual_error(nlh_net net, const nlh_net_batch *batch, double *e0,
                                  void *stream);

/* Loss of the batch (HOST double; NULL to skip the copy, which keeps the
 * call asynchronous) and its gradient with respect to every parameter,
 * kept in the network for nlh_net_adam / nlh_net_get_grads. */
nlh_status nlh_net_loss_grad(nlh_net net, const nlh_net_batch *batch, double *loss,
                             void *stream);

/* One Adam step with the stored gradient:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * Stream-ordered. */
nlh_status nlh_net_adam(nlh_net net, double lr, double beta1, double beta2, double eps,
                        void *stream);

/* Engine of the 3x3 forward and input-gradient convolutions (implicit
 * GEMMs, bf16 operands, f32 accumulation):
 *   NLH_NET_ENGINE_TCGEN05  (default) 5th-generation tensor cores, the
 *                           accumulator in tensor memory;
 *   NLH_NET_ENGINE_MMA_SYNC warp-level mma.sync (register accumulators).
 * Both sum the same products per 32-channel chunk; results agree to f32
 * rounding order.  Errors: NLH_ERR_ARG. */
enum { NLH_NET_ENGINE_MMA_SYNC = 0, NLH_NET_ENGINE_TCGEN05 = 1 };
nlh_status nlh_net_set_engine(nlh_net net, int engine);
nlh_status nlh_net_get_engine(nlh_net net, int *engine);

/* Synchronise `stream` and report NLH_ERR_TIMEOUT if a bounded wait inside
 * a tensor-core kernel gave up since the last check (the outputs of the
 * calls in between are then invalid; the word is cleared).  The synchronous
 * calls (get_params, get_grads, loss_grad with a loss pointer) check too. */
nlh_status nlh_net_check(nlh_net net, void *stream);

/* Free the network (NULL is a no-op). */
nlh_status nlh_net_destroy(nlh_net net);

/* Degrees d = Gamma_full 1 of a plan in pixel order (DEVICE N doubles),
 * from its most accurate NFFT arithmetic (FP64, else double-float, else
 * FP32): the input of the Jacobi diagonal P_a = alpha + max(d - 1, 0).
 * Stream-ordered. */
nlh_status nlh_plan_get_degrees(nlh_plan plan, double *d, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NLH_NET_H */
