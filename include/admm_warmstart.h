/*
 * admm_warmstart.h -- learned starting point for the ADMM deconvolution solver.
 *
 * The paper has no learned component. Its Theorem 1 makes Algorithm 2
 * converge from any (u0, d0); this library exploits that with a small
 * convolutional network that predicts a starting image x0 and duals d0 from
 * the observation, which admm_deconv_warm_start (admm_deconv.h) turns into
 * the start u0 = H x0 - d0. The solver then runs to its usual stop rule, so
 * the plain ADMM still decides the result.
 *
 * Network: 8 convolutions of 3 x 3 (zero padding, "same" size), 32 channels,
 * ReLU between them:
 *     input  [M^T y, mask]   2 channels
 *     output o               4 channels, no activation
 * The start is x0 = s0 o0, d1 = s1 o1, d2 = (s2 o2, s2 o3) (TV duals).
 * Weights and activations are BF16, products accumulate in FP32 on the
 * tensor cores; master weights, gradients and Adam moments are FP32.
 *
 * Parameter vector (FP32, admm_cnn_param_count() floats): for each layer in
 * order, the weights w[cout][cin][3][3] (row-major; w[o][i][p+1][q+1]
 * multiplies input channel i at offset (p, q)) and then the biases b[cout].
 *
 * All image arguments hold `count` images of H x W pixels back to back
 * (device memory). H and W must be multiples of 16, at least 16.
 * Every call returns 0 (ADMM_OK) or a negative admm status code.
 */
#ifndef ADMM_WARMSTART_H
#define ADMM_WARMSTART_H

#include <stdint.h>

#include "admm_deconv.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ADMM_CNN_LAYERS 8
#define ADMM_CNN_WIDTH 32

typedef struct admm_cnn_s* admm_cnn_t;

/* Number of FP32 parameters of the network (57252). */
ADMM_API long long admm_cnn_param_count(void);

/*
 * admm_cnn_create -- allocate a network for batches of up to `max_pixels`
 * pixels in total (count x H x W). training = 1 also allocates what
 * admm_cnn_train_step and admm_cnn_gradients need (stored activations,
 * gradients, Adam moments: about 0.7 KB per pixel); 0 keeps inference only.
 * Parameters start at zero: set them with admm_cnn_set_params.
 * Errors: ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA.
 */
ADMM_API int admm_cnn_create(admm_cnn_t* out, long long max_pixels, int training);

/* Copy the FP32 parameter vector in (host or device); resets Adam's state. */
ADMM_API int admm_cnn_set_params(admm_cnn_t net, const float* params);

/* Copy the FP32 parameter vector out (host or device). */
ADMM_API int admm_cnn_get_params(admm_cnn_t net, float* params);

/*
 * admm_cnn_forward -- network output for `count` observations.
 *   ybar  count x H x W float32: observed values (ignored where mask = 0)
 *   mask  count x H x W uint8: 1 = observed
 *   out   count x H x W x 4 float32: the four output channels per pixel
 */
ADMM_API int admm_cnn_forward(admm_cnn_t net, int count, int H, int W, const float* ybar,
                              const uint8_t* mask, float* out, void* stream);

/*
 * admm_cnn_gradients -- loss and its gradient in every parameter, without
 * updating them. Loss = mean over images and pixels of
 * sum_k chan_w[k] (o_k - target_k)^2, with target count x H x W x 4 float32
 * (device) and chan_w 4 floats (host).
 *   grads  admm_cnn_param_count() floats (device or host), parameter layout
 *   loss   host, may be NULL
 * Requires a network created with training = 1.
 */
ADMM_API int admm_cnn_gradients(admm_cnn_t net, int count, int H, int W, const float* ybar,
                                const uint8_t* mask, const float* target, const float* chan_w,
                                float* grads, double* loss, void* stream);

/*
 * admm_cnn_train_step -- one Adam step (beta1 0.9, beta2 0.999, eps 1e-8,
 * step size lr) on the loss of admm_cnn_gradients over this batch.
 * loss (host, may be NULL) receives the loss before the step; with NULL the
 * call does not wait for the device.
 */
ADMM_API int admm_cnn_train_step(admm_cnn_t net, int count, int H, int W, const float* ybar,
                                 const uint8_t* mask, const float* target, const float* chan_w,
                                 float lr, double* loss, void* stream);

/*
 * admm_cnn_predict_start -- the warm start of `count` TV problems:
 *   scales  4 floats (host): s0, s1, s2 (s3 unused)
 *   x0      count x H x W float32 (device): s0 o0
 *   d0      count x 3 H W float32 (device), per image in the layout of
 *           admm_deconv_get_state for TV: d1 = s1 o1 (H x W), then
 *           (s2 o2, s2 o3) interleaved per pixel
 * Pass x0 + i H W and d0 + 3 i H W to admm_deconv_warm_start.
 */
ADMM_API int admm_cnn_predict_start(admm_cnn_t net, int count, int H, int W, const float* ybar,
                                    const uint8_t* mask, const float* scales, float* x0, float* d0,
                                    void* stream);

/* Kernels launched by this part of the library since it was loaded. */
ADMM_API long long admm_cnn_launches(void);

ADMM_API void admm_cnn_destroy(admm_cnn_t net);

#ifdef __cplusplus
}
#endif

#endif /* ADMM_WARMSTART_H */
