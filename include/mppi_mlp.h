/*
 * mppi_mlp.h - learned proposal for the MPPI update (C ABI).
 *
 * The paper samples around the previous plan (Sec. II) with the strategy of
 * another paper (Sec. III-B).  This layer adds a learned proposal: an MLP
 * maps (q, qd, goal, current nominal plan) to the plan that plain MPPI would
 * produce, and the update samples around that prediction.  The network is
 *   x (n_in) -> [Linear -> GELU] x n_layers (width n_hidden) -> Linear (n_out)
 * with BF16 weights and activations and FP32 accumulation on the tensor
 * cores (tcgen05.mma into tensor memory, operands staged by TMA), FP32
 * master weights and Adam.  Inputs and outputs are standardised with fixed
 * per-feature means and deviations.
 * The loss is the mean squared error of the standardised outputs.
 * Parameters are flat FP32: W_1 [n_hidden][n_in] row-major, b_1, W_2, b_2,
 * ..., W_L [n_out][n_hidden], b_L.  All device pointers are caller-owned
 * FP32 arrays; work is queued on the stream given at creation.
 */
#ifndef MPPI_MLP_H
#define MPPI_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "mppi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mppi_mlp_s* mppi_mlp_t;

typedef struct mppi_mlp_config {
  int n_in, n_hidden, n_layers, n_out;  /* n_layers hidden layers, 1..6; widths <= 1024 */
  int max_batch;                        /* rows per forward / train step, 1..65536      */
  uint64_t seed;                        /* weight initialisation                         */
  float beta1, beta2, eps;              /* Adam                                          */
} mppi_mlp_config;

/* Creates the network on the current device with Kaiming-uniform weights,
 * zero biases, identity standardisation.  stream: cudaStream_t or NULL. */
MPPI_API int mppi_mlp_create(const mppi_mlp_config* cfg, void* stream, mppi_mlp_t* out);
MPPI_API int mppi_mlp_destroy(mppi_mlp_t m);
MPPI_API int mppi_mlp_num_params(mppi_mlp_t m, size_t* n);
/* FP32 master parameters (host arrays of num_params floats); set also
 * refreshes the BF16 copies and clears the Adam moments. */
MPPI_API int mppi_mlp_get_params(mppi_mlp_t m, float* host);
MPPI_API int mppi_mlp_set_params(mppi_mlp_t m, const float* host);
/* Per-feature standardisation (host arrays; deviations must be > 0). */
MPPI_API int mppi_mlp_set_normalization(mppi_mlp_t m, const float* mean_in, const float* std_in,
                                        const float* mean_out, const float* std_out);
/* The standardisation fitted to training data on the device: per-feature
 * means and deviations (unbiased, FP64 sums) of d_x [n][n_in] and d_y
 * [n][n_out], deviations below floor raised to it (floor > 0, n >= 2);
 * blocks until done. */
MPPI_API int mppi_mlp_fit_normalization(mppi_mlp_t m, const float* d_x, const float* d_y, int n,
                                        float floor);
/* y = net(x) for n rows of raw inputs d_x [n][n_in]; raw outputs d_y [n][n_out]. */
MPPI_API int mppi_mlp_forward(mppi_mlp_t m, const float* d_x, int n, float* d_y);
/* Loss and gradient for n rows (d_y: raw targets); grad_host (num_params
 * floats, may be NULL) receives the gradient; blocks until done. */
MPPI_API int mppi_mlp_loss_grad(mppi_mlp_t m, const float* d_x, const float* d_y, int n,
                                float* loss, float* grad_host);
/* One Adam step (learning rate lr) on n rows; *loss (may be NULL: no wait)
 * receives the batch loss before the step.  The calls that wait (loss_grad,
 * train_step with a loss) return MPPI_ERR_TIMEOUT if a tensor-core GEMM
 * gave up waiting for its operands (a bounded wait; the work is skipped). */
MPPI_API int mppi_mlp_train_step(mppi_mlp_t m, const float* d_x, const float* d_y, int n,
                                 float lr, float* loss);
/* Learned proposal for an MPPI handle: x = (q, qd, goal from d_in [25
 * device floats], the handle's current nominal plan u [T][7]); the network
 * predicts the correction that plain MPPI would make to u, and u + net(x)
 * is installed as the second proposal of the handle's next update with
 * n_plain samples kept around the plain warm start (mppi_set_proposal_device;
 * n_plain = 0 samples only around the network's plan).  One launch of a
 * cluster of 8 CTAs, queued on the handle's stream; it reads the network's
 * weights, which a training step must not be changing at the same time.
 * Needs n_in = 21 + 7T and n_out = 7T, at most 3 hidden layers and widths
 * <= 256 (MPPI_ERR_INVALID_ARG otherwise). */
MPPI_API int mppi_mlp_propose(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain);
/* mppi_mlp_propose followed by mppi_step_device(h, d_in, d_tau0, d_plan) in
 * one call: the update runs with the proposal it installs.  The two are
 * queued back to back, and on the plain warp-specialised rollout kernel
 * (variant 3 without the optional costs) the update's blocks whose samples
 * all lie below n_plain start while the proposal is still being formed
 * (programmatic dependent launch); the other blocks wait for it.  The
 * result is the same, bit for bit, as the two calls made one after the
 * other.  Errors as for the two calls, the message of either in
 * mppi_last_error(NULL); nothing is queued when the proposal's arguments
 * are rejected. */
MPPI_API int mppi_mlp_propose_step_device(mppi_mlp_t m, mppi_t h, const float* d_in, int n_plain,
                                          float* d_tau0, float* d_plan);
/* The timeout path of the bounded device waits: one mbarrier wait that
 * nothing completes, given up after `cycles` SM clock cycles (1 ..
 * about 2e9, the limit of the GEMMs' own waits) through the same helper and
 * error flag; blocks until done and returns MPPI_ERR_TIMEOUT (clearing the
 * flag), MPPI_ERR_INVALID_ARG for a bad argument.  The paper has no
 * counterpart. */
MPPI_API int mppi_mlp_check_wait(mppi_mlp_t m, long long cycles);

#ifdef __cplusplus
}
#endif

#endif /* MPPI_MLP_H */
