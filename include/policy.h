/*
 * policy.h -- C ABI of the closed-loop policy MLP and its gradient (sm_103a
 * CUDA, tensor cores), for backpropagation through time of a policy acting
 * on the simulator's own observations (Sec. IV: the learners' MLP backbone;
 * Eq. 5: the gradient flows through the simulator's adjoint).
 *
 * Per agent (rigid body, one agent per environment):
 *   obs = (p - p*, q, v, omega, p [16], depth * (1/cam_range) [Rc],
 *          lidar * (1/lidar_range) [Rl])                  F = 16 + Rc + Rl
 *   x   = bf16(obs)
 *   h   = bf16(silu(W1 x + b1))                           256
 *   a   = tanh(W2 h + b2)                                 4 actions in (-1, 1)
 * W1, W2 rounded to bf16 for the products, fp32 accumulation (tcgen05 for
 * the K = F layer).  Parameters (HOST, pol_nparams floats): W1 [256][F],
 * b1 [256], W2 [4][256], b2 [4], row-major.
 *
 * pol_act keeps what its backward pass needs (inputs, pre-activations,
 * actions); pol_backward takes the action cotangent (from sim_step_backward),
 * accumulates the parameter gradient in the handle and returns the
 * observation cotangent split into state, depth and LiDAR parts, so the
 * caller can chain it into the previous step's adjoint.
 *
 * Conventions as in diffsim.h (SIM_OK / SIM_ERR_*; DEVICE pointers are the
 * caller's CUDA buffers used on the given stream; HOST pointers are read or
 * written synchronously).
 */
#ifndef POLICY_H
#define POLICY_H

#include "diffsim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pol_handle pol_handle;

#define POL_HIDDEN 256
#define POL_ACTIONS 4
#define POL_STATE_FEATURES 16

/* n_env agents; cam_rays / lidar_rays (0: no such sensor) and the ranges
 * that normalise them (> 0 when the sensor exists).  Parameters start at
 * zero, the gradient accumulator at zero. */
int pol_create(int32_t n_env, int32_t cam_rays, float cam_range, int32_t lidar_rays, float lidar_range,
               pol_handle **out);
int pol_destroy(pol_handle *h); /* NULL-safe */

int pol_nparams(const pol_handle *h, int64_t *n);
int pol_set_params(pol_handle *h, const float *params); /* HOST; keeps the gradient accumulator */
int pol_get_params(pol_handle *h, float *params);       /* HOST */

/* Actions [N][4] (DEVICE) of states [N][13], targets [N][3], depth [N][Rc]
 * and lidar [N][Rl] (DEVICE; a sensor's pointer may be NULL when it has no
 * rays). */
int pol_act(pol_handle *h, const float *state, const float *targets, const float *depth, const float *lidar,
            float *actions, sim_stream_t stream);

/* Backward pass of the last pol_act: g_actions [N][4] (DEVICE).  Adds the
 * parameter gradient to the handle's accumulator; adds the state part of the
 * observation cotangent to g_state [N][13] (DEVICE, read and updated);
 * writes the depth and LiDAR parts to g_depth [N][Rc] and g_lidar [N][Rl]
 * (DEVICE, nullable when the sensor has no rays).  SIM_ERR_NOT_READY before
 * a pol_act. */
int pol_backward(pol_handle *h, const float *g_actions, float *g_state, float *g_depth, float *g_lidar,
                 sim_stream_t stream);

/* Copies the accumulated gradient (pol_nparams floats) to grads (HOST,
 * synchronises); reset != 0 zeroes the accumulator afterwards. */
int pol_grads(pol_handle *h, float *grads, int32_t reset);

/* Status word since the last call (2: a bounded wait gave up); synchronises. */
int pol_last_status(pol_handle *h, int32_t *status);

#ifdef __cplusplus
}
#endif

#endif /* POLICY_H */
