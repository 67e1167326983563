/* The warm-start network: a per-interface fully connected GELU network that proposes each
 * interface's initial dual variables for the next time step (the learned warm start of the
 * ADMM loop, Algorithm 1, in place of the previous step's duals of Sec. III-D).  The paper
 * has no such component; its method only fixes what the network replaces (z^0, u^0 = -lambda^0).
 *
 * Numerics: weights are FP32 masters with BF16 copies; the layers compute in BF16 with FP32
 * accumulation on the tensor cores; hidden activations are stored in BF16, pre-activations
 * and outputs in FP32.  GELU is the exact form u Phi(u).
 *
 * Pointers named *_dev are device pointers (stream-ordered on `stream`, a cudaStream_t, NULL
 * for the legacy stream); all others are host pointers, copied during the call.  The handle
 * owns its device memory.  Negative returns are errors (SIM_E* codes of subadmm.h), the
 * message in wsn_last_error.  One host thread per handle.
 */
#ifndef WARMSTART_H
#define WARMSTART_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wsn_s *wsn_t;

/* A network of n_layers layers with widths sizes[0] (input) .. sizes[n_layers] (output),
 * each at most 1024; on `device`.  Parameters start at zero (set them with wsn_set_params). */
int wsn_create(int device, int n_layers, const int *sizes, wsn_t *out);
void wsn_destroy(wsn_t w);
const char *wsn_last_error(wsn_t w);

/* Number of parameters: sum over layers of in x out + out. */
long long wsn_num_params(wsn_t w);

/* shape[0] the input width, shape[1] the output width. */
int wsn_shape(wsn_t w, int shape[2]);

/* Identifies the network's current activation workspace: unique within the process, it
 * changes whenever a call with a larger batch than before reallocates the workspace.  A
 * caller that captured wsn_forward into a CUDA graph must recapture when it changes. */
long long wsn_workspace_generation(wsn_t w);

/* Parameters in layer order: W_1 (in x out, row-major: W[i * out + j] maps input i to
 * output j), b_1, W_2, b_2, ...  Setting also refreshes the BF16 copies and resets Adam. */
int wsn_set_params(wsn_t w, const float *params);
int wsn_get_params(wsn_t w, float *params);

/* Input normalisation and output scale (host arrays): the network sees
 * (x - mean_in) / std_in and its outputs are multiplied by scale_out at inference.  Defaults:
 * 0, 1 and 1. */
int wsn_set_normalization(wsn_t w, const float *mean_in, const float *std_in,
                          const float *scale_out);
int wsn_get_normalization(wsn_t w, float *mean_in, float *std_in, float *scale_out);

/* Fit the normalisation on training data (device): mean_in and std_in per input column of
 * x (batch rows, leading dimension ldx; a column with std < 1e-6 gets std 1), and
 * scale_out per output column as the root mean square of t (1 where that is 0). */
int wsn_fit_normalization(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                          int batch, void *stream);

/* Inference: y (batch x out, FP32) = scale_out * net((x - mean_in) / std_in).  For the
 * warm-start shape (32 -> 256 -> 256 -> 256 -> 7) all four layers run in one fused launch on
 * the tcgen05 tensor cores (the BF16 weights packed K-major on every call, activations in
 * shared memory between layers, accumulators in tensor memory); other shapes run layer by
 * layer.  Both compute the same arithmetic (BF16 weights and activations, FP32 accumulation,
 * exact GELU) and differ only in the order of the FP32 sums. */
int wsn_forward(wsn_t w, const float *x_dev, long long ldx, int batch, float *y_dev,
                void *stream);

/* The layer-by-layer inference (one tensor-core GEMM launch per layer) for any shape: the
 * reference the fused path is tested against. */
int wsn_forward_layers(wsn_t w, const float *x_dev, long long ldx, int batch, float *y_dev,
                       void *stream);

/* Reads and clears the fused inference kernel's error word: *out = 1 if one of its waits
 * ran out (1 s) since the last call (its outputs are then undefined).  Synchronous. */
int wsn_fused_error(wsn_t w, int *out);

/* Gradients of the masked mean-squared loss L = sum mask (net(x) - t / scale_out)^2 / (2 batch)
 * (the targets t in output units, divided by scale_out inside), written to grad_dev in the
 * parameter order of wsn_set_params; the loss is added to *loss_dev (may be NULL). */
int wsn_gradients(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                  const float *mask_dev, int batch, float *grad_dev, float *loss_dev,
                  void *stream);

/* One Adam step (bias-corrected, beta1 0.9, beta2 0.999, eps 1e-8) on the gradients of a
 * minibatch; the loss of the minibatch is added to *loss_dev (may be NULL). */
int wsn_train_step(wsn_t w, const float *x_dev, long long ldx, const float *t_dev,
                   const float *mask_dev, int batch, float lr, float *loss_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif
