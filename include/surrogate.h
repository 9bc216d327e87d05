/* Learned seismogram surrogate of libsemgb: an MLP and a 1D-convolution decoder that map a
 * source (location and moment tensor) to the three-component traces of the receivers of one
 * fixed medium, trained on runs of the spectral-element solver (include/sem.h). The
 * surrogate is not in arXiv 2606.12850; the solver it is trained on follows Sec. II-B and
 * Sec. V-C of the paper, and the solver stays the fallback and the measure of its error.
 *
 * Network (all sizes fixed at sg_create):
 *   h1 = gelu(x W1^T + b1)            in_dim -> hidden
 *   h2 = gelu(h1 W2^T + b2)           hidden -> hidden
 *   z  = gelu(h2 W3^T + b3)           hidden -> c0 * l0, viewed as [c0][l0]
 *   stage s = 0 .. nstages-1:         z = act(conv3(up_s(z)) + c_s)
 * up_s repeats every time sample up[s] times (1 or 2), conv3 is the zero-padded width-3
 * cross-correlation over all input channels, act = gelu (tanh form) except for the last
 * stage (identity). With contract = K > 0 the last stage has K * C channels D and the
 * output is y[c][t] = sum_k x[in_dim - K + k] D[k*C + c][t]: linear in the last K inputs
 * (the moment-tensor entries, in which seismograms are linear). Output y: float32
 * [batch][C][l0 * prod(up)], C = cout[nstages-1] / K (or cout[nstages-1] when K = 0).
 * Loss: mean squared error over all outputs.
 *
 * Precision: float32 master parameters; every weight product (dense layers, convolutions
 * and their backward products) runs on the tensor cores with bfloat16 operands (the
 * bfloat16 copies of the weights, activations and gradients rounded to nearest even) and
 * float32 accumulation; biases, activations, the loss and the moment contraction stay
 * float32. Adam (Kingma and Ba 2015) updates the master parameters and refreshes the
 * bfloat16 copies.
 *
 * Parameter order (every host array of parameters or gradients is this concatenation,
 * float32): W1 [hidden][in_dim], b1 [hidden], W2 [hidden][hidden], b2 [hidden],
 * W3 [c0*l0][hidden], b3 [c0*l0], then per stage C_s [cout_s][cin_s][3], c_s [cout_s]
 * with cin_0 = c0 and cin_s = cout_{s-1}.
 *
 * Ownership and errors as in sem.h: host pointers are used during the call only; *_dev
 * pointers are device arrays on the model's GPU, borrowed until the model's stream reaches
 * the end of the call. Calls return SG_OK (0) or a negative code (the SEM_* values) and
 * leave a message for sg_last_error. A model is not thread-safe.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_OK 0
#define SG_MAX_STAGES 8

typedef struct sg_model sg_model;

/* Create a model on device `device`, working on `stream` (a cudaStream_t, or NULL for a
 * stream of its own). stage_cout[nstages] and stage_up[nstages] (1 or 2) describe the
 * decoder; max_batch bounds the batch of sg_loss_grad (sg_forward runs larger batches in
 * chunks of max_batch), and max_batch x the output length must be below 2^24. Parameters
 * start at zero (set them with sg_set_params). */
int sg_create(sg_model** out, int device, void* stream, int in_dim, int hidden, int c0, int l0, int nstages,
              const int32_t* stage_cout, const int32_t* stage_up, int contract, int max_batch);
int sg_destroy(sg_model* model);

/* Sizes: out[0] parameter count, out[1] output channels, out[2] output length,
 * out[3] bytes of device memory held. */
int sg_info(sg_model* model, int64_t* out);

/* Master parameters from / to a host float32 array in the parameter order above. */
int sg_set_params(sg_model* model, const float* params);
int sg_get_params(sg_model* model, float* params);

/* y_dev[batch][cout][L] = network(x_dev[batch][in_dim]). Asynchronous on the stream. */
int sg_forward(sg_model* model, int batch, const float* x_dev, float* y_dev);

/* Forward and backward pass on one batch (batch <= max_batch): the gradient of the mean
 * squared error against target_dev[batch][cout][L] is left in the model (see
 * sg_get_grads) and the loss, accumulated in float64, is written to *loss (host).
 * Synchronous. */
int sg_loss_grad(sg_model* model, int batch, const float* x_dev, const float* target_dev, double* loss);
int sg_get_grads(sg_model* model, float* grads);

/* One Adam step with the gradients of the last sg_loss_grad (bias-corrected, step count
 * kept by the model), then bfloat16 copies of the weights refreshed. Asynchronous. */
int sg_adam_step(sg_model* model, float lr, float beta1, float beta2, float eps);

int sg_sync(sg_model* model);

/* Options. SG_OPT_PRODUCT picks the kernel of every product (dense layers, convolutions and
 * their backward products): 1 (the default) = tcgen05.mma with the float32 accumulator in
 * tensor memory, 128 x 128 tiles (the convolutions stage their input window once for the
 * three taps); 0 = warp-level mma.sync, 128/256 x 64 tiles. Both round the
 * operands to bfloat16 and accumulate in float32, so they agree to float32 rounding order.
 * Setting an option waits for the model's stream. A tcgen05 product that waits more than 2 s
 * for its MMAs gives up: sg_loss_grad and sg_sync then return SEM_ETIMEOUT. */
#define SG_OPT_PRODUCT 1
/* SG_OPT_STALL_TEST (tests only): 1 makes every tcgen05 product wait for an mbarrier phase
 * that nothing completes, with a 20 ms limit that runs out; the next sg_loss_grad or sg_sync returns
 * SEM_ETIMEOUT, no result of the product is written and the model stays usable. */
#define SG_OPT_STALL_TEST 2
int sg_set_option(sg_model* model, int option, int value);
int sg_get_option(sg_model* model, int option, int* value);
const char* sg_last_error(const sg_model* model);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_H */
