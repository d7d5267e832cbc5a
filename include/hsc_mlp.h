/* hsc_mlp.h -- surrogate network of the learned energy grid (libhsc.so).
 *
 * A fully connected network x (n_in) -> [Linear -> GELU] x hidden_layers (width) -> Linear -> y
 * (n_out), GELU(z) = 0.5 z (1 + tanh(sqrt(2/pi)(z + 0.044715 z^3))), trained with mean-squared
 * error and Adam on the GPU. It predicts log T(E) and DOS(E) from E and disorder features so that an
 * adaptive energy grid can concentrate points where they vary fastest; every integrated quantity is
 * still computed by hsc_solve on that grid. The paper has no learned component.
 *
 * Parameters (float32, host layout for set/get): for each layer l: W_l (d_in x d_out, row-major,
 * y = x W + b) followed by b_l (d_out). x, y, t are device float32 arrays [batch][n_in|n_out].
 * All calls return an hsc_status; hsc_last_error(NULL) gives text.
 */
#ifndef HSC_MLP_H
#define HSC_MLP_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsc_mlp_ctx* hsc_mlp_t;

/* allocate parameters (zero), Adam moments and activations for up to max_batch rows */
int hsc_mlp_create(hsc_mlp_t* out, int32_t n_in, int32_t width, int32_t hidden_layers,
                   int32_t n_out, int32_t max_batch);
int hsc_mlp_num_params(hsc_mlp_t m, int64_t* n);
/* host float32 parameters in the layout above; set also resets Adam's moments and step */
int hsc_mlp_set_params(hsc_mlp_t m, const float* host);
int hsc_mlp_get_params(hsc_mlp_t m, float* host);
/* y = net(x); bf16 = 1 reads a BF16 copy of the parameters (FP32 accumulation) */
int hsc_mlp_forward(hsc_mlp_t m, int32_t batch, const float* x, float* y, int32_t bf16,
                    void* cuda_stream);
/* forward + mean-squared-error loss against t + backward; gradients stay on the device for
 * hsc_mlp_adam; loss_host / grad_host (num_params floats) are optional host copies (the call then
 * synchronises the stream) */
int hsc_mlp_loss_grad(hsc_mlp_t m, int32_t batch, const float* x, const float* t, float* loss_host,
                      float* grad_host, void* cuda_stream);
/* one Adam step with the last gradients (bias-corrected moments) */
int hsc_mlp_adam(hsc_mlp_t m, float lr, float beta1, float beta2, float eps, void* cuda_stream);
int hsc_mlp_destroy(hsc_mlp_t m);

#ifdef __cplusplus
}
#endif
#endif
