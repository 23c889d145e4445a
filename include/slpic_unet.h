/*
 * slpic_unet.h -- C ABI of the small convolutional U-Net that supplies the
 * initial guess of the 2D field solve (slpic2d.h, slpic2d_set_warm_start).
 *
 * The paper leaves the field solve of Eq. (LimPtclDynAppendixDotE) unchanged
 * from plain PIC and has no learned part.  Here a network maps the charge
 * density rho of the 2D grid to a guess of phi; the conjugate-gradient solve to
 * the same relative residual stays the judge of the answer, so the guess changes
 * the work, not the result (up to the solver's tolerance).
 *
 * Network, level l = 0..L-1 with C_l = C * 2^l channels at (H/2^l) x (W/2^l):
 *   encoder  e_0 = relu(conv(x)),  e_l = relu(conv(pool(e_{l-1})))
 *   decoder  d_{L-1} = e_{L-1},    d_l = relu(conv(concat(up(d_{l+1}), e_l)))
 *   output   y = conv(d_0)                                      (1 channel)
 * conv: 3x3, zero padding, stride 1, with bias; pool: 2x2 mean; up: nearest
 * x2; concat: the channels of up(d_{l+1}) first, then those of e_l.
 *
 * Scaling.  With normalise != 0 each sample n is divided by its RMS
 * s_n = sqrt(mean(x_n^2)) (1 for an all-zero sample) before the network, and the
 * output is multiplied by s_n * out_scale.  phi depends linearly on rho (zero
 * plate potentials), so one network then serves every charge amplitude.  With
 * normalise == 0, s_n = 1.  The training target t is compared with the network
 * output in network units, t / (s_n * out_scale).
 *
 * Precision: activations and gradients FP32; the convolutions multiply by a
 * BF16 copy (round to nearest even) of the FP32 master weights and accumulate in
 * FP32; biases FP32; weight-gradient sums FP64 across threads; loss sums FP64.
 * With tensor_cores = 1 the forward convolutions and the input-gradient
 * convolutions run as implicit GEMMs on the tensor cores (tcgen05, BF16 x BF16,
 * FP32 accumulate in tensor memory, output channels in slices of 256): each
 * forward conv's input is rounded to BF16 (nearest even), and the weight gradient
 * multiplies by that rounded input; the input gradient is the transposed conv of
 * the output gradient rounded to BF16, and passes the forward rounding through
 * unchanged; the weight gradient is a GEMM over the pixels (split over CTAs, the
 * parts added in a fixed order) of the rounded input and the rounded output
 * gradient; the bias gradient sums the unrounded output gradient in FP64.
 *
 * Parameters: one flat FP32 array, conv by conv in the order encoder
 * l = 0..L-1, decoder l = L-2..0, output; each conv its weights
 * W[c_out][c_in][3][3] (row-major) followed by its biases b[c_out].
 * Initialisation: He-normal weights, N(0, 2 / (9 c_in)), from a SplitMix64
 * stream seeded with `seed` and Box-Muller; zero biases.
 *
 * Training loss, with e = y_net - t_net and count = nb * H * W:
 *   SLPIC_UNET_LOSS_MSE     L = sum e^2 / count;
 *   SLPIC_UNET_LOSS_ENERGY  L = sum_n (e_n . A e_n) / count, the energy norm of
 *       the error under the 2D field solve's 5-point operator A (slpic2d.h) on
 *       the image read as that solver's grid: row 0 a plate, the other plate
 *       just past row H-1, both at zero; columns periodic; e zeroed on row 0;
 *       A e = 4 e - e(x+-1) - e(y+-1).  The conjugate-gradient solve's error
 *       falls in this norm, so it is the measure of a guess.
 * Adam (Kingma & Ba, 2015) with bias correction on the FP32 master weights.
 *
 * Arrays: x, y, t are DEVICE pointers to nb * H * W FP32 values (sample-major,
 * row-major (H, W) per sample); calls on them are asynchronous on the handle's
 * stream.  Parameter and gradient copies (set/get_params, gradients' grads) are
 * HOST arrays and synchronise.  The forward activations are allocated by
 * slpic_unet_create; the gradient buffers by the first slpic_unet_gradients or
 * slpic_unet_train_step call (SLPIC_ERR_OOM if that fails), so an inference-only
 * handle holds none.  Return codes, error strings and handle ownership are those
 * stated at the top of slpic.h.
 */
#ifndef SLPIC_UNET_H
#define SLPIC_UNET_H

#include "slpic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slpic_unet slpic_unet_t;

#define SLPIC_UNET_LOSS_MSE 0
#define SLPIC_UNET_LOSS_ENERGY 1

typedef struct {
    int32_t levels;        /* L >= 1                                                 */
    int32_t base;          /* C >= 1: channels of level 0                             */
    int32_t height, width; /* H, W >= 1, both divisible by 2^(L-1); H*W <= 2^28       */
    int32_t max_batch;     /* samples per call, >= 1 (activation buffers sized for it)*/
    int32_t normalise;     /* per-sample RMS scaling of input and output (see above)  */
    int32_t loss;          /* SLPIC_UNET_LOSS_MSE or SLPIC_UNET_LOSS_ENERGY           */
    int32_t tensor_cores;  /* 1: convolutions forward on the tensor cores (below)     */
    double out_scale;      /* output factor (> 0)                                     */
    double adam_beta1;     /* 0 -> 0.9                                                */
    double adam_beta2;     /* 0 -> 0.999                                              */
    double adam_eps;       /* 0 -> 1e-8                                               */
    uint64_t seed;         /* initialisation stream                                   */
} slpic_unet_config;

int slpic_unet_create(const slpic_unet_config *cfg, slpic_unet_t **out);
int slpic_unet_destroy(slpic_unet_t *h);
const char *slpic_unet_last_error(slpic_unet_t *h);
/* Stream (cudaStream_t) for the calls below; NULL = the legacy default stream. */
int slpic_unet_set_stream(slpic_unet_t *h, void *stream);

/* Number of FP32 parameters (weights and biases of every conv). */
int slpic_unet_param_count(slpic_unet_t *h, int64_t *n);
/* Copy the master parameters in (refreshing the BF16 copy) or out: HOST arrays
 * of slpic_unet_param_count values in the order stated above. */
int slpic_unet_set_params(slpic_unet_t *h, const float *params);
int slpic_unet_get_params(slpic_unet_t *h, float *params);

/* y = network(x) with the scaling above, for nb (1..max_batch) samples. */
int slpic_unet_forward(slpic_unet_t *h, int32_t nb, const float *x, float *y);

/* Forward, loss and backward for nb samples against targets t.  *loss (may be
 * NULL) receives the mean squared error in network units; grads (HOST, may be
 * NULL) receives dL/dparams in the parameter order.  Leaves the parameters
 * alone.  Synchronises when loss or grads is non-NULL. */
int slpic_unet_gradients(slpic_unet_t *h, int32_t nb, const float *x, const float *t,
                         double *loss, float *grads);

/* One Adam step of learning rate lr on the gradients of nb samples.  *loss (may
 * be NULL: no synchronisation) receives the loss before the step. */
int slpic_unet_train_step(slpic_unet_t *h, int32_t nb, const float *x, const float *t,
                          double lr, double *loss);

/* Zero Adam's moments and step count (the parameters stay). */
int slpic_unet_reset_optimizer(slpic_unet_t *h);

#ifdef __cplusplus
}
#endif

#endif
