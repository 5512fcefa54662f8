/*
 * bandred_tune: the learned cost model of the band-reduction autotuner.
 *
 * Section 4.2 of the paper shows that the best algorithmic block size b depends on n, w
 * and the parallelism, and tunes b by timing for every problem dimension and bandwidth.
 * The library keeps that search (paper_1709_00302_gb300.tune times candidate
 * configurations through the bandred_*_ex calls) and adds a small regression model that
 * predicts log run time from a configuration's features, so that only the best-ranked
 * candidates of an untimed size class need to be timed.  The paper has no counterpart of
 * the model; it only ranks configurations and never changes a result.
 *
 * Model: a multilayer perceptron with two tanh hidden layers of width H,
 *     h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = w3 . h2 + b3,
 * in FP32, with every parameter in one flat device array, in this order and layout:
 *     W1  H x D, row-major (W1[h * D + d])
 *     b1  H
 *     W2  H x H, row-major (W2[h * H + g], weight of h1[g] in unit h)
 *     b2  H
 *     w3  H
 *     b3  1
 * 1 <= D <= 32 inputs, 1 <= H <= 64 hidden units.  Inputs X are row-major, rows x D.
 * Loss: mean squared error L = (1/rows) sum_r (y_r - t_r)^2.
 * Optimiser: Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization", 2015,
 * Algorithm 1) with bias correction.
 *
 * All pointers are device memory owned by the caller; calls are stream-ordered, never
 * allocate and never synchronise.  Every sum over rows runs in a fixed order, so results
 * are bitwise reproducible on one GPU.  Return value: 0, or -i when argument i is
 * invalid, or BANDRED_ERR_CUDA (include/bandred.h) when a launch failed.
 */
#ifndef BANDRED_TUNE_H
#define BANDRED_TUNE_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of FP32 parameters of a D-input, H-hidden model: H*D + H + H*H + H + H + 1. */
size_t bandred_mlp_param_count(int d_in, int hidden);

/* Bytes of device workspace bandred_mlp_loss_grad needs for `rows` rows. */
size_t bandred_mlp_workspace(int d_in, int hidden, int rows);

/* y[r] = model(X[r, :]) for r < rows. */
int bandred_mlp_forward(int d_in, int hidden, const float* params, const float* X, int rows, float* y,
                        cudaStream_t stream);

/* grad (param_count floats) = dL/dparams and *loss = L (one float, device) for the
 * targets t[rows]; work holds the per-row activations and deltas. */
int bandred_mlp_loss_grad(int d_in, int hidden, const float* params, const float* X, const float* t, int rows,
                          float* grad, float* loss, void* work, size_t work_bytes, cudaStream_t stream);

/* One Adam step on `count` parameters: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).  step >= 1. */
int bandred_mlp_adam(int count, float* params, const float* grad, float* m, float* v, int step, float lr,
                     float beta1, float beta2, float eps, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BANDRED_TUNE_H */
