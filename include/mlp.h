/*
 * mlp.h - C ABI of the surrogate network used to propose wall couplings.
 *
 * The network maps the parameters of a capillary run to observables that the
 * lattice Boltzmann model measures: inputs (G_Aw, G_Bw, G_AB, tau_A, tau_B,
 * H) and outputs (cos theta, Washburn prefactor, precursor prefactor), after
 * the caller's normalisation.  The paper maps contact angle to wall coupling
 * only a posteriori, by simulation (Model section, after Eq. 11); the
 * network is a fast stand-in for that map, and every proposal it makes is
 * checked by running the lattice model.
 *
 * Architecture: fully connected 6 -> 128 -> 128 -> 128 -> 3, exact GELU
 * (x Phi(x), erf form) between layers, linear output.  Parameters are one
 * FP32 vector of MLP_N_PARAMS values in layer order W1, b1, W2, b2, W3, b3,
 * W4, b4, W_l stored [in][out] row-major (y = x W + b).  GEMM operands are
 * bfloat16 (weights and layer inputs rounded to nearest even), products are
 * accumulated in FP32 on the tensor cores (mma.sync m16n8k16); biases,
 * activations and the optimiser state stay FP32.  Training minimises the mean
 * squared error over batch and outputs with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on FP32 master weights.
 *
 * Conventions: return 0 (MLP_OK) or a positive error code; x, t, y, grad and
 * loss pointers are device pointers of the current device owned by the
 * caller; all work is asynchronous on the stream given at creation
 * (NULL = legacy default stream).  A handle is not thread-safe.
 */
#ifndef SHANCHEN_GB300_MLP_H
#define SHANCHEN_GB300_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLP_OK 0
#define MLP_EINVAL 1   /* bad argument (n < 1 or above max_batch, NULL pointer) */
#define MLP_ENOMEM 2   /* device allocation failed */
#define MLP_ECUDA 3    /* a CUDA call failed */

#define MLP_N_IN 6
#define MLP_N_HIDDEN 128
#define MLP_N_OUT 3
#define MLP_N_PARAMS 34307

typedef struct mlp_s mlp_t;

/* Creates a network for batches of up to max_batch rows.  params: host FP32
 * [MLP_N_PARAMS] initial weights (NULL = all zero).  Allocates the
 * parameters, the Adam moments and the per-batch activation scratch. */
int mlp_create(int max_batch, const float* params, void* stream, mlp_t** out);

/* Replaces the parameters (host FP32 [MLP_N_PARAMS]) and resets the Adam
 * moments and step count.  Synchronises. */
int mlp_set_params(mlp_t* h, const float* params);

/* Copies the FP32 master parameters to host params[MLP_N_PARAMS].  Synchronises. */
int mlp_get_params(mlp_t* h, float* params);

/* y[n][3] = network(x[n][6]) for 1 <= n <= max_batch. */
int mlp_forward(mlp_t* h, const float* x, int n, float* y);

/* Gradient of the loss mean((y - t)^2) with respect to the parameters,
 * grad[MLP_N_PARAMS], and the loss itself (loss[1]), for targets t[n][3].
 * The batch reductions run in a fixed order: repeated calls give identical
 * bits. */
int mlp_gradients(mlp_t* h, const float* x, const float* t, int n, float* grad, float* loss);

/* One training step: forward, backward, Adam update with learning rate lr,
 * refresh of the bfloat16 weights.  loss (nullable) receives the loss of the
 * batch before the update. */
int mlp_train_step(mlp_t* h, const float* x, const float* t, int n, float lr, float* loss);

/* Number of Adam steps taken since creation or the last mlp_set_params. */
int64_t mlp_step_count(const mlp_t* h);

/* Frees the handle's device memory.  NULL is a no-op. */
void mlp_destroy(mlp_t* h);

#ifdef __cplusplus
}
#endif
#endif /* SHANCHEN_GB300_MLP_H */
