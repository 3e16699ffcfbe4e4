/*
 * surrogate.h -- C ABI of the learned surrogate of the rigid-body step
 * (sm_103a CUDA, tensor cores).
 *
 * A residual MLP stands in for one explicit step of the rigid quadrotor
 * (Eq. 1), the learned-dynamics model that the paper's world-model learners
 * (Sec. IV) fit to simulator transitions:
 *     x  = (s [13], clip(a, -1, 1) [4]),  xh = (x - mu_x) * rs_x
 *     y  = W3 silu(W2 silu(W1 xh + b1) + b2) + b3          17 -> 256 -> 256 -> 13
 *     s' = s + (sd_d * y + mu_d), quaternion renormalised
 * bf16 weights and activations, fp32 accumulation (tcgen05, accumulators in
 * tensor memory).  Training: mean squared error of y against the normalised
 * residual t = ((s1 - s) - mu_d) * rs_d, Adam.  Where an environment's inputs
 * leave the range seen in training (each feature within [lo - m, hi + m],
 * m = margin * (hi - lo)), the rollout takes the plain rigid-body step of the
 * simulator instead.
 *
 * Conventions as in diffsim.h: SIM_OK or a negative SIM_ERR_* code; DEVICE
 * pointers are the caller's CUDA buffers used on the given stream; HOST
 * pointers are read or written synchronously.  Layouts are row-major.
 *   parameters  SURR_NPARAM floats: W1 [256][17], b1 [256], W2 [256][256],
 *               b2 [256], W3 [13][256], b3 [13]
 *   statistics  SURR_NSTATS floats: mu_x [17], rs_x [17], lo_x [17],
 *               hi_x [17], mu_d [13], sd_d [13], rs_d [13]
 *   transitions X [n][17] (state, action), S1 [n][13] (next state)
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include "diffsim.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SURR_NIN 17
#define SURR_NHID 256
#define SURR_NOUT 13
#define SURR_NPARAM 73741
#define SURR_NSTATS 107

typedef struct surr_handle surr_handle;

typedef struct surr_config {
    int32_t batch;       /* training minibatch: a multiple of 128, 128 .. 262144 */
    int32_t splits;      /* split-K factor of the weight gradients (0: automatic) */
    float lr, beta1, beta2, eps;  /* Adam (1e-3, 0.9, 0.999, 1e-8) */
    float margin;        /* trained-range margin, fraction of (hi - lo) (0.1) */
    int32_t reserved[5]; /* zero */
} surr_config;

/* Creates a handle on the current device.  phys (HOST): a rigid-body
 * configuration (model SIM_MODEL_RIGID) whose dt, gravity, mass, inertia,
 * k_rate, drag_body and rate_scale define the plain step.  Parameters start
 * at zero; statistics at mu = 0, rs = sd = 1, an unbounded range. */
int surr_create(const surr_config *cfg, const sim_config *phys, surr_handle **out);
int surr_destroy(surr_handle *h); /* NULL-safe */

/* Parameters (HOST, SURR_NPARAM floats).  Setting them resets Adam's moments
 * and step count and re-packs the bf16 copies. */
int surr_set_params(surr_handle *h, const float *params);
int surr_get_params(surr_handle *h, float *params);

/* Statistics (HOST, SURR_NSTATS floats). */
int surr_set_stats(surr_handle *h, const float *stats);
int surr_get_stats(surr_handle *h, float *stats);

/* Statistics of a transition set (DEVICE X [n][17], S1 [n][13]) computed on
 * the GPU and kept in the handle: means, 1 / standard deviations (1 where the
 * deviation is below 1e-6) and ranges of the inputs (actions clipped), mean,
 * deviation and its inverse of the residuals s1 - s. */
int surr_fit_stats(surr_handle *h, const float *X, const float *S1, int64_t n, sim_stream_t stream);

/* Network outputs y [n][13] (DEVICE) of raw inputs X [n][17] (DEVICE). */
int surr_forward(surr_handle *h, const float *X, int64_t n, float *Y, sim_stream_t stream);

/* One Adam step on the minibatch rows idx [batch] (DEVICE int32, each in
 * [0, n)) of the transition set X, S1.  loss (DEVICE float, nullable): the
 * minibatch mean squared error before the update.  grads (DEVICE
 * SURR_NPARAM floats, nullable): the gradient.  apply = 0 computes loss and
 * gradient and leaves parameters and moments untouched. */
int surr_train_step(surr_handle *h, const float *X, const float *S1, const int32_t *idx, float *loss,
                    float *grads, int32_t apply, sim_stream_t stream);

/* T surrogate steps of N environments from s0 [N][13] under actions
 * [T][N][4] (DEVICE).  states [T+1][N][13], sT [N][13] and fallback [T][N]
 * (1 where the plain step was taken) are DEVICE outputs, each nullable. */
int surr_rollout(surr_handle *h, const float *s0, const float *actions, int32_t N, int32_t T, float *states,
                 float *sT, uint8_t *fallback, sim_stream_t stream);

/* Status word of the kernels since the last call (1 non-finite state, 2 a
 * bounded wait gave up); synchronises the last stream and clears it. */
int surr_last_status(surr_handle *h, int32_t *status);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_H */
