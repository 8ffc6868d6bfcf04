/*
 * esp_mlp.h - the small network of the learned parameter selector: a 3-layer perceptron
 * trained and evaluated on the GPU by the library's own kernels (FP32).
 *
 * The paper tunes ESP by analytic rules (Sec. 5.1: psi_0(1) = Delta for the split and the
 * spreading, P = ceil(-log10 Delta) + 1, the grid from the cut-off |k| <= c / r_c); it has
 * no learned component.  This network maps features of a system and an accuracy target to
 * ESP parameters; the selector built on it (paper_2601_00161_gb300/selector.py) falls
 * back to the analytic rules.
 *
 * Network: a1 = W1 x + b1, h1 = tanh(a1); a2 = W2 h1 + b2, h2 = tanh(a2); y = W3 h2 + b3.
 * Loss: mean squared error over the batch and the outputs.  Parameters form one FP32
 * vector in the order W1 (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2,
 * W3 (n_out x n_hidden), b3.  Optimiser: Adam with bias correction.
 *
 * All device pointers are float arrays the caller owns; batches are row-major
 * (batch x n_in inputs, batch x n_out targets / outputs).  Calls are asynchronous on the
 * stream given at creation.  Return codes: 0 on success, ESP_ERR_ARG (-1) for bad
 * arguments, ESP_ERR_CUDA (-6) for CUDA failures; esp_mlp_last_error describes the last one.
 */
#ifndef ESP_MLP_H
#define ESP_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esp_mlp_s* esp_mlp_t;

/* Number of parameters of a network of these sizes. */
int esp_mlp_n_params(int n_in, int n_hidden, int n_out);

/* Create a network (device parameters copied from params_host, esp_mlp_n_params floats)
 * with workspace for batches of up to max_batch rows; Adam moments start at zero. */
int esp_mlp_create(esp_mlp_t* out, int n_in, int n_hidden, int n_out, int max_batch,
                   const float* params_host, void* stream);

/* Inference: y (batch x n_out) from x (batch x n_in), device arrays. */
int esp_mlp_forward(esp_mlp_t net, const float* d_x, int batch, float* d_y);

/* Forward and back-propagation on a batch: d_loss (1 float, device) receives the mean
 * squared error; the gradient is kept for esp_mlp_adam and, if d_grad is not NULL, copied
 * to it (esp_mlp_n_params floats, device). */
int esp_mlp_loss_grad(esp_mlp_t net, const float* d_x, const float* d_t, int batch,
                      float* d_loss, float* d_grad);

/* One Adam step with the last gradient (step counter kept by the network). */
int esp_mlp_adam(esp_mlp_t net, float lr, float beta1, float beta2, float eps);

/* Copy the parameters from / to host memory (esp_mlp_n_params floats); synchronous. */
int esp_mlp_get_params(esp_mlp_t net, float* params_host);
int esp_mlp_set_params(esp_mlp_t net, const float* params_host);

int esp_mlp_destroy(esp_mlp_t net);
const char* esp_mlp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif
