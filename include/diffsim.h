/*
 * diffsim.h -- C ABI of the fused, batched, differentiable quadrotor
 * environment step (DiffAero, arXiv 2509.10247), sm_103a CUDA.
 *
 * One handle simulates N environments of M agents each.  Per step it
 * integrates one of the four dynamics models (Eq. 1-4), ray-casts the depth
 * camera and / or LiDAR against the environment's spheres, axis-aligned
 * boxes, vertical cylinders and racing-gate frames (Sec. III-B), reads the
 * IMU, evaluates collisions, the differentiable reward R_ctrl and the sparse
 * reward R_goal of the reaching / avoidance or racing task (Sec. III-C,
 * III-D, III-E), terminates and resets environments, and renders the new
 * observation.  A rollout of T steps is two launches (the sequential physics
 * of all T steps, then every step's ray casting); its adjoint
 * (backpropagation through time, Eq. 5) is hand-written, also two launches.
 * A reset + rollout + adjoint can be captured once into a CUDA graph.
 *
 * Conventions
 *  - Every function returns SIM_OK (0) or a negative SIM_ERR_* code; no C++
 *    exception crosses this boundary.  sim_strerror() names a code.
 *  - "device" pointers are CUDA global memory of the handle's device, owned
 *    by the caller, read or written asynchronously on the given stream; the
 *    caller keeps them alive until the stream has passed the call.  "host"
 *    pointers are read synchronously and may be freed on return.
 *  - Floating point is FP32 everywhere on the device.  Layouts are row-major
 *    with the last index fastest:
 *      state    [NM][D]   NM = N*M; D = 12 point mass, continuous and discrete
 *                          (p[3], v[3], a[3], ema_v[3]; for the discrete
 *                          model a is the thrust acceleration in force);
 *                          D = 13 rigid (p[3], q[4] = (w,x,y,z), v[3],
 *                          omega[3]); D = 15 simplified (p[3], v[3], R[9]
 *                          row-major body -> world)
 *      actions  [T][NM][A]  A = 3 point mass (acceleration command), 4 rigid
 *                          and simplified (thrust, 3 body rates), each in
 *                          [-1, 1] (clipped)
 *      r_ctrl   [T][NM] float, r_goal [T][NM] int8, done [T][NM] uint8
 *      depth    [T][NM][Rc], Rc = cam_w * cam_h, ray = row * cam_w + col
 *      lidar    [T][NM][Rl], Rl = lid_ch * lid_az, ray = ch * lid_az + k
 *    Output t of a rollout is the observation of the state after step t.
 *  - A handle is not thread safe; calls on one handle must be ordered.
 */
#ifndef DIFFSIM_H
#define DIFFSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t-compatible opaque stream (NULL = legacy default stream) */
typedef struct CUstream_st *sim_stream_t;
typedef struct sim_handle sim_handle;

enum {
    SIM_OK = 0,
    SIM_ERR_INVALID_ARG = -1, /* a value out of its documented range */
    SIM_ERR_NULL_PTR = -2,    /* a required pointer is NULL */
    SIM_ERR_SIZE = -3,        /* sizes inconsistent or beyond a limit */
    SIM_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    SIM_ERR_NOT_READY = -5,   /* e.g. step before set_scene, backward before rollout */
    SIM_ERR_NAN = -6,         /* a non-finite state was produced (status word) */
    SIM_ERR_TIMEOUT = -7,     /* a bounded device wait gave up (status word) */
    SIM_ERR_OOM = -8,         /* device allocation failed */
    SIM_ERR_UNSUPPORTED = -9  /* no kernel for this configuration */
};

/* Dynamics models (Sec. III-A): continuous point mass (Eq. 3), full rigid
 * body (Eq. 1), discrete point mass (Eq. 4), simplified quadrotor (Eq. 2). */
enum { SIM_MODEL_POINT_MASS = 0, SIM_MODEL_RIGID = 1, SIM_MODEL_POINT_MASS_DISCRETE = 2, SIM_MODEL_SIMPLE = 3 };

/* Status bits accumulated on the device (sim_last_status). */
enum { SIM_STATUS_NAN = 1, SIM_STATUS_TIMEOUT = 2, SIM_STATUS_MAP_CAPACITY = 4 };

/* Simulation parameters.  Paper symbols: Eq. 3 (lam, drag), Eq. 1 (mass,
 * inertia J, drag_body D), Sec. III-B (sensors), Sec. III-C/D/E (task). */
typedef struct sim_config {
    int32_t model;        /* SIM_MODEL_* */
    int32_t n_env;        /* N >= 1 */
    int32_t n_agent;      /* M >= 1 agents per environment (swarm) */
    int32_t horizon;      /* T >= 1 steps per rollout */
    float dt;             /* step length (s) */
    float gravity;        /* |g| (m/s^2), acting along world -z */
    /* continuous point mass, Eq. 3 */
    float lam;            /* command latency factor lambda (1/s) */
    float drag;           /* drag coefficient d (1/s) */
    float act_scale;      /* acceleration command u = act_scale * clip(a) (m/s^2) */
    float ema_alpha;      /* velocity EMA weight of the point-mass heading */
    /* rigid body, Eq. 1, with rate controller tau = J K (w_c - w) + w x J w */
    float mass;           /* kg */
    float inertia[3];     /* diagonal of J (kg m^2) */
    float k_rate[3];      /* diagonal of K (1/s) */
    float drag_body[3];   /* diagonal of D (1/s) */
    float rate_scale[3];  /* body-rate command w_c = rate_scale * clip(a1..3) (rad/s) */
    /* depth camera (cam_w = 0: none): pinhole along +x_B, z-depth output */
    int32_t cam_w, cam_h;
    float cam_hfov;       /* horizontal field of view (rad) */
    float cam_range;      /* z-depth clamp (m) */
    /* LiDAR (lid_ch = 0: none): range output */
    int32_t lid_ch, lid_az;
    float lid_elev_lo, lid_elev_hi; /* channel elevations (rad), inclusive */
    float lid_range;      /* range clamp (m) */
    /* task / reward */
    int32_t pos_sq;       /* 1: -w_pos |e|^2 (position task); 0: -w_pos |e| */
    float w_pos, w_obs, d_safe, w_act, w_agent, d_agent, success_radius, r_quad;
    float bound_lo[3], bound_hi[3]; /* leaving this box is a collision (+-inf: none) */
    int32_t terminate;    /* 1: a collision ends the env's episode and resets it */
    int32_t pool_size;    /* P reset states per agent (sim_set_pool) */
    /* execution */
    int32_t ckpt_every;   /* K: rollout checkpoints every K steps (0: K = T) */
    int32_t tape_hits;    /* 1: rollout stores ray hit ids, backward gathers them;
                             0: backward re-casts the rays; -1: auto (tape if <= 8 GiB) */
    int32_t cull;         /* field-of-view culling (result-preserving): 0 off, 1 per sensor
                             frustum, 2 frustum and per ray-chunk cones, -1 auto (cones
                             when a 128-ray chunk's cone is on average under half the
                             sensor's own, ray-weighted: large images, LiDAR scans) */
    int32_t warps_per_cta;   /* 0: auto (8); else warps per CTA, 1..8 */
    int32_t rays_per_thread; /* 0: auto (4 with cones, else the best lane fill); else one
                                of 1, 2, 3, 4, 5, 6, 8 */
    int32_t ctas_per_sm;     /* 0: occupancy limit; else cap of resident CTAs per SM */
    /* flight task (Sec. III-C): SIM_TASK_REACH (targets; position control and
       obstacle avoidance) or SIM_TASK_RACING (the map's gates in order; needs
       at least one gate in every map) */
    int32_t task;
    /* IMU noise (Sec. III-B), used when noise samples are given: white-noise
       standard deviation of the specific force (m/s^2) and angular rate
       (rad/s), and the standard deviation per sqrt(s) of their bias random
       walks; all >= 0 */
    float imu_noise[2], imu_walk[2];
    int32_t cast_mode;       /* execution: 0 thread per ray (each lane sweeps the cull list for
                                its rays); 1 warp per ray (the lanes split the list and a
                                warp-level min-reduction picks the nearest hit; maps of spheres
                                and boxes only, others cast thread per ray).  Same results bit
                                for bit */
} sim_config;

/* Flight tasks. */
enum { SIM_TASK_REACH = 0, SIM_TASK_RACING = 1 };

/* Library version string. */
const char *sim_version(void);

/* Human-readable name of an error code (static storage). */
const char *sim_strerror(int code);

/* State dimension D and action dimension A of a model; -1 for an unknown model. */
int sim_state_dim(int model);
int sim_action_dim(int model);

/* Create a handle on the current CUDA device.  Validates cfg (every count
 * positive, horizon >= 1, camera and LiDAR sizes, tape/cull flags, launch
 * knobs) and allocates the state, checkpoints, tapes and ray tables.
 * *out is NULL on failure.  The handle owns its device memory. */
int sim_create(const sim_config *cfg, sim_handle **out);

/* Free a handle and its device memory (synchronises the device first).
 * NULL is a no-op. */
int sim_destroy(sim_handle *h);

/* Bytes of device memory the handle holds (state, checkpoints, tapes, scene). */
int sim_workspace_bytes(const sim_handle *h, size_t *bytes);

/* Obstacle scene (Sec. III-B, III-C), all HOST pointers, copied in
 * synchronously:
 *   spheres [Ks][4] = (cx, cy, cz, r), boxes [Kb][6] = (min xyz, max xyz);
 *   sph_off, box_off [n_maps + 1]: map m owns spheres sph_off[m] ..
 *   sph_off[m+1]-1 and boxes box_off[m] .. box_off[m+1]-1 (at most 32767
 *   primitives per map; within a map spheres take ids 0..ns-1, boxes ns..);
 *   env_map [N]: map of each environment; targets [NM][3]: goal positions.
 * Errors: NULL_PTR, SIZE (offsets not non-decreasing, an env_map entry out
 * of range, a map too large for shared memory), INVALID_ARG (radius or box
 * extent negative, non-finite values). */
int sim_set_scene(sim_handle *h, const float *spheres, const int32_t *sph_off,
                  const float *boxes, const int32_t *box_off, int32_t n_maps,
                  const int32_t *env_map, const float *targets);

/* Scene with all four primitive kinds (HOST pointers, copied in).  Each kind
 * has a CSR offset array [n_maps + 1]; a kind's array may be NULL with its
 * offsets NULL (none of that kind).  Within a map, ids run over spheres,
 * boxes, cylinders, gates in that order (at most 32767 in total), ties of
 * the ray cast go to the lowest id.
 *   cylinders [Kc][5] = (cx, cy, r, zmin, zmax): vertical (axis along world
 *     z), capped; r >= 0, zmin <= zmax
 *   gates [Kg][7] = (cx, cy, cz, yaw, w, b, hd): a square frame around an
 *     open square of half-width w, border width b, half-depth hd along its
 *     normal (cos yaw, sin yaw, 0); w, b, hd > 0.  In the racing task the
 *     map's gates are the course, passed in id order along their normals.
 * Errors as sim_set_scene; SIZE also when the racing task meets a map
 * without gates. */
typedef struct sim_scene {
    int32_t n_maps;
    const float *spheres;
    const int32_t *sph_off;
    const float *boxes;
    const int32_t *box_off;
    const float *cylinders;
    const int32_t *cyl_off;
    const float *gates;
    const int32_t *gate_off;
    const int32_t *env_map; /* [N] */
    const float *targets;   /* [NM][3] (ignored by the racing task) */
} sim_scene;

int sim_set_scene_ex(sim_handle *h, const sim_scene *scene);

/* Racing: each agent's index of the next gate [NM] (DEVICE int32), read or
 * set.  sim_reset sets every index to 0; a reset of an environment sets its
 * agents' indices to 0; passing the targeted gate advances it cyclically. */
int sim_get_gate_index(const sim_handle *h, int32_t *gate_k, sim_stream_t stream);
int sim_set_gate_index(sim_handle *h, const int32_t *gate_k, sim_stream_t stream);

/* Reset pool [P][NM][D], HOST pointer, P = cfg.pool_size: on termination
 * environment e takes entry (k_e mod P) for all its agents, k_e counting
 * its resets.  Required when terminate = 1. */
int sim_set_pool(sim_handle *h, const float *pool);

/* Per-environment drag d and latency lambda (Sec. IV-D domain
 * randomisation), HOST pointers [N] each, either may be NULL (= cfg value). */
int sim_set_env_params(sim_handle *h, const float *drag, const float *lam);

/* Set the current state from a DEVICE buffer [NM][D] and zero the reset
 * counters.  state0 = NULL takes pool entry 0. */
int sim_reset(sim_handle *h, const float *state0, sim_stream_t stream);

/* Copy the current state to / from a DEVICE buffer [NM][D]. */
int sim_get_state(const sim_handle *h, float *dst, sim_stream_t stream);
int sim_set_state(sim_handle *h, const float *src, sim_stream_t stream);

/* Copy the per-environment reset counters to / from a DEVICE int32 [N]: the
 * k of the pool entry (k mod P) the environment takes at its next reset
 * (Sec. IV-A resets; sim_reset zeroes them).  With sim_get/set_state they
 * make a checkpoint from which steps replay bit for bit. */
int sim_get_reset_counters(const sim_handle *h, int32_t *dst, sim_stream_t stream);
int sim_set_reset_counters(sim_handle *h, const int32_t *src, sim_stream_t stream);

/* Sensor outputs of the current state (the initial observation): depth
 * [NM][Rc] and lidar [NM][Rl], DEVICE, either NULL to skip. */
int sim_render(sim_handle *h, float *depth, float *lidar, sim_stream_t stream);

/* sim_render that also records, per ray, the primitive its depth comes from
 * (Sec. III-B ray casting; the ray term of the Eq. 5 adjoint needs only that
 * primitive): hits_cam [NM][Rc] and hits_lidar [NM][Rl], int16 DEVICE,
 * caller-owned; -1 = no hit within range, -2 = the sensor's origin lies
 * inside a primitive (depth 0, no gradient).  Either may be NULL (that
 * sensor's hits are not written).  Feeds sim_step_backward_taped of the step
 * that produced this state, which then gathers the hits instead of casting
 * every ray again (closed loop: the backward pass re-renders state t for
 * the policy anyway; its hits serve the adjoint of step t-1). */
int sim_render_taped(sim_handle *h, float *depth, float *lidar, int16_t *hits_cam,
                     int16_t *hits_lidar, sim_stream_t stream);

/* Depth [NM][Rc] and lidar [NM][Rl] (DEVICE, either NULL to skip) of the
 * current state from hit ids recorded for that state (sim_render_taped or
 * sim_step_ex): each ray evaluates only its recorded primitive with the
 * cast's own arithmetic, so the images equal sim_render's bit for bit at a
 * fraction of the cost (no culling, no search).  Hits of another state
 * give wrong images but stay memory-safe (ids outside the environment's map
 * read as misses).  A sensor with an output needs its hits (else
 * SIM_ERR_NULL_PTR).  Lets a closed loop keep every step's hits (2 bytes
 * per ray) instead of casting each observation again in its backward pass. */
int sim_render_hits(sim_handle *h, const int16_t *hits_cam, const int16_t *hits_lidar, float *depth,
                    float *lidar, sim_stream_t stream);

/* One step of the current state with actions [NM][A] (DEVICE).  Outputs
 * (DEVICE, any may be NULL): depth [NM][Rc], lidar [NM][Rl], r_ctrl [NM],
 * r_goal [NM], done [NM].  Advances the current state. */
int sim_step(sim_handle *h, const float *actions, float *depth, float *lidar,
             float *r_ctrl, int8_t *r_goal, uint8_t *done, sim_stream_t stream);

/* T = cfg.horizon steps from the current state in one persistent launch.
 * actions [T][NM][A]; outputs r_ctrl [T][NM], r_goal [T][NM], done [T][NM],
 * depth [T][NM][Rc], lidar [T][NM][Rl] (DEVICE, any may be NULL).  Records
 * checkpoints (and hit tapes) for sim_backward and advances the state. */
int sim_rollout(sim_handle *h, const float *actions, float *r_ctrl, int8_t *r_goal,
                uint8_t *done, float *depth, float *lidar, sim_stream_t stream);

/* Inputs and outputs of one rollout (sim_rollout_ex) or one step
 * (sim_step_ex, T = 1), DEVICE pointers, any output NULL to skip:
 *   actions [T][NM][A]; r_ctrl, r_goal, done [T][NM]; depth [T][NM][Rc],
 *   lidar [T][NM][Rl] as in sim_rollout;
 *   imu [T][NM][6]: the IMU readout of the state after each step (Sec.
 *     III-B) in the body frame: specific force f = R^T (v' - g) of the
 *     model's translational dynamics (rigid: (T/m) e3 - D R^T v; point mass:
 *     R^T (a - d v); discrete: R^T u; simplified: c e3), then the angular
 *     rate (rigid: the state's omega; simplified: the commanded rates; point
 *     mass: the attitude change over the step, vee(A - A^T) / (2 dt),
 *     A = R_t^T R_{t+1}); after a reset the new state read at rest
 *     (-R^T g, the rigid rate state, else 0);
 *   imu_noise [T][NM][12] (nullable): standard normal samples, 6 white-noise
 *     terms added with the cfg.imu_noise deviations and 6 steps of the bias
 *     random walk (cfg.imu_walk * sqrt(dt)); the bias starts at 0 at
 *     sim_reset and at every reset of an environment. */
typedef struct sim_rollout_io {
    const float *actions;
    float *r_ctrl;
    int8_t *r_goal;
    uint8_t *done;
    float *depth, *lidar;
    float *imu;
    const float *imu_noise;
    /* sim_step_ex only (sim_rollout_ex: must be NULL, SIM_ERR_INVALID_ARG):
     * per-ray hit ids of the rendered state as sim_render_taped writes them,
     * [NM][Rc] / [NM][Rl] int16, nullable */
    int16_t *hits_cam, *hits_lidar;
} sim_rollout_io;

int sim_rollout_ex(sim_handle *h, const sim_rollout_io *io, sim_stream_t stream);
int sim_step_ex(sim_handle *h, const sim_rollout_io *io, sim_stream_t stream);

/* Cotangents and gradients of the adjoint, DEVICE pointers (inputs NULL =
 * zero): g_r [T][NM], g_depth [T][NM][Rc], g_lidar [T][NM][Rl], g_sT
 * [NM][D], g_imu [T][NM][6] (the IMU readout; the noise is additive and
 * passes no cotangent); outputs g_a [T][NM][A], g_s0 [NM][D] (nullable). */
typedef struct sim_grad_io {
    const float *g_r, *g_depth, *g_lidar, *g_sT, *g_imu;
    float *g_a, *g_s0;
} sim_grad_io;

int sim_backward_ex(sim_handle *h, const sim_grad_io *io, sim_stream_t stream);

/* Adjoint of the last sim_rollout (Eq. 5): given cotangents g_r [T][NM] of
 * r_ctrl, g_depth [T][NM][Rc], g_lidar [T][NM][Rl] and g_sT [NM][D] of the
 * final state (DEVICE; g_depth, g_lidar, g_sT may be NULL = zero), writes
 * g_a [T][NM][A] and g_s0 [NM][D] (g_s0 may be NULL).  No cotangent crosses
 * a reset; kinks take the active branch's derivative.  The actions buffer
 * given to sim_rollout must still hold the same values.
 * Errors: NOT_READY without a preceding rollout. */
int sim_backward(sim_handle *h, const float *g_r, const float *g_depth, const float *g_lidar,
                 const float *g_sT, float *g_a, float *g_s0, sim_stream_t stream);

/* Vector-Jacobian product of one step (closed-loop use; the reaching task
 * only, SIM_ERR_UNSUPPORTED for racing): state s_t [NM][D],
 * actions a_t [NM][A], done_t [NM] (the step's done output), cotangents
 * g_s_next [NM][D] (may be NULL), g_r [NM], g_depth [NM][Rc], g_lidar
 * [NM][Rl] (may be NULL); outputs g_a [NM][A], g_s [NM][D] (may be NULL).
 * All DEVICE.  Re-casts the rays of the step; does not touch the current state. */
int sim_step_backward(sim_handle *h, const float *s_t, const float *a_t, const uint8_t *done_t,
                      const float *g_s_next, const float *g_r, const float *g_depth,
                      const float *g_lidar, float *g_a, float *g_s, sim_stream_t stream);

/* sim_step_backward whose ray adjoint gathers hit ids instead of re-casting:
 * hits_cam [NM][Rc], hits_lidar [NM][Rl] (int16, DEVICE) written by
 * sim_render_taped of the state this step produces (s_t stepped with a_t).
 * Each sensor with a non-NULL cotangent needs its hits (SIM_ERR_NULL_PTR
 * otherwise); both hits NULL = sim_step_backward.  Ids from another state
 * give a wrong gradient but stay memory-safe (ids outside the environment's
 * map are ignored).  The result equals sim_step_backward's bit for bit when
 * the hits match the step. */
int sim_step_backward_taped(sim_handle *h, const float *s_t, const float *a_t,
                            const uint8_t *done_t, const float *g_s_next, const float *g_r,
                            const float *g_depth, const float *g_lidar, const int16_t *hits_cam,
                            const int16_t *hits_lidar, float *g_a, float *g_s,
                            sim_stream_t stream);

/* Device status word accumulated by the kernels since the last call
 * (SIM_STATUS_* bits; synchronises the handle's last stream and clears it).
 * per_env is reserved and must be NULL. */
int sim_last_status(sim_handle *h, int32_t *status, int32_t *per_env);

/* sim_set_wait_limit: polls > 0 limits the first wait of every render and
 * rollout CTA of h (the wait for its map's bulk copy) to that many
 * non-blocking polls; 0 (the default) restores the full bounded wait.  The
 * paper has no counterpart: this exercises the failure path of the bounded
 * device waits.  A wait that runs out sets SIM_STATUS_TIMEOUT; the CTA then
 * waits (fully bounded) for its copy in flight and stops, so the launch's
 * outputs are incomplete and sim_last_status returns SIM_ERR_TIMEOUT, while
 * the handle and the CUDA context stay usable.  SIM_ERR_INVALID_ARG for
 * polls < 0. */
int sim_set_wait_limit(sim_handle *h, int32_t polls);

/* Work counters accumulated by the forward kernels since the last reset:
 * out[0] ray-sphere tests, out[1] ray-box tests (both after field-of-view
 * culling), out[2] rays cast, out[3] environment steps.  Synchronises the
 * last stream.  reset != 0 zeroes the counters after reading. */
int sim_counters(sim_handle *h, uint64_t *out, int32_t reset);

/* Whether the forward kernels of h count their work (on != 0, the default)
 * into the counters that sim_counters reads; with 0 they skip the counting
 * atomics (a few shared-memory atomics per 32 x rays-per-thread ray slots),
 * for timing runs that take the counts from a separate counted pass.  Takes
 * effect at the next launch; SIM_ERR_NULL_PTR for a null handle. */
int sim_set_counting(sim_handle *h, int32_t on);

/* sim_fp32_issue_rate: measures this GPU's FP32 multiply-add rate, the
 * denominator of the ray cast's roofline (the paper has no counterpart: a
 * measurement utility).  Runs a grid of 8 CTAs of 256 threads per SM, each
 * thread 8 independent FMA chains, timed with CUDA events on `stream` (the
 * call synchronises it); the fastest of three passes after a warm-up.
 *   scratch        DEVICE float[scratch_floats] that receives the chains'
 *                  sums (>= 2048 * SM count floats, else SIM_ERR_SIZE)
 *   fma_per_s      HOST out: scalar FMAs per second (one FP32-pipe
 *                  instruction per lane and FMA)
 *   ffma2_per_s    HOST out (nullable): FMAs per second issued as packed
 *                  pairs (one instruction per lane, two FMAs) */
int sim_fp32_issue_rate(float *scratch, int64_t scratch_floats, double *fma_per_s, double *ffma2_per_s,
                        sim_stream_t stream);

/* Bytes of the library's static device scratch used by sim_step_static. */
#define SIM_STATIC_SCRATCH_BYTES (256 * 1024)

/* sim_step_static: one step, like sim_step, that allocates no device memory
 * (reaching task, spheres and boxes, no IMU: cfg.task must be SIM_TASK_REACH).
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc (code that must draw all device memory from a pool
 * or arena owned by someone else, or that has fixed its allocations up
 * front): they pass every buffer, and the step's scratch (work ticket,
 * status word, counters, camera / LiDAR ray tables) lives in one static
 * device array of SIM_STATIC_SCRATCH_BYTES that every GPU which loads the
 * library holds until the process exits.  Limit: 20 * (Rc + Rl) + 64 bytes
 * must fit in it (at most 13104 rays per agent), else SIM_ERR_SIZE.
 *   cfg      simulation parameters (HOST); execution fields warps_per_cta,
 *            rays_per_thread and cull are honoured, the others ignored
 *   prims    DEVICE, the scene in the library's layout: per map a block of
 *            float4, map_ns[m] spheres (cx, cy, cz, r) followed by map_nb[m]
 *            boxes as (min x, y, z, 0), (max x, y, z, 0); 16-byte aligned
 *   map_off, map_ns, map_nb  DEVICE [n_maps]: block start (in float4),
 *            sphere and box counts; ns_max, nb_max: their maxima (HOST ints)
 *   env_map [N], targets [NM][3], pool [P][NM][D] (NULL: no reset)  DEVICE
 *   state    DEVICE [NM][D], read and overwritten with the next state
 *   actions  DEVICE [NM][A]; outputs depth, lidar, r_ctrl, r_goal, done as
 *            in sim_step (any may be NULL); pool_k DEVICE [N] reset counters
 *            (read and advanced; NULL: entry 0 and no counting)
 *   status   DEVICE int32 (nullable): receives this call's SIM_STATUS_* bits
 *            once the step has run on `stream` (no host synchronisation):
 *            SIM_STATUS_NAN a non-finite state, SIM_STATUS_TIMEOUT a bounded
 *            wait for the map copy gave up (that environment was skipped),
 *            SIM_STATUS_MAP_CAPACITY a map with more spheres or boxes than
 *            ns_max / nb_max (checked on the device before staging; the
 *            environments of that map are left untouched: outputs unwritten,
 *            state unchanged).  Read it before relying on the outputs.
 * The first call on a device looks up the scratch address on that device
 * (again whenever the device's context has changed, e.g. after
 * cudaDeviceReset); make it before any stream capture.  Every call rewrites
 * the scratch, so calls that overlap on the GPU (other streams, other
 * threads) race; order them on one stream.  Returns SIM_OK or a SIM_ERR_*
 * code. */
int sim_step_static(const sim_config *cfg, const float *prims, const int32_t *map_off,
                    const int32_t *map_ns, const int32_t *map_nb, int32_t ns_max, int32_t nb_max,
                    const int32_t *env_map, const float *targets, const float *pool, float *state,
                    const float *actions, float *depth, float *lidar, float *r_ctrl,
                    int8_t *r_goal, uint8_t *done, int32_t *pool_k, int32_t *status,
                    sim_stream_t stream);

/* Launch shape chosen for this handle: warps per CTA, rays per thread,
 * grid size of the rollout kernel and its dynamic shared memory (bytes). */
int sim_launch_info(const sim_handle *h, int32_t *warps_per_cta, int32_t *rays_per_thread,
                    int32_t *grid, int32_t *smem_bytes);

/* Kernel kinds counted and timed by the library. */
enum {
    SIM_KERNEL_PHYSICS = 0,     /* sequential dynamics, collisions, rewards, resets, poses */
    SIM_KERNEL_RENDER = 1,      /* ray casting of camera / LiDAR for every step */
    SIM_KERNEL_RENDER_VJP = 2,  /* ray adjoint: depth / range cotangent -> pose cotangent */
    SIM_KERNEL_PHYSICS_BWD = 3, /* physics adjoint over checkpointed segments */
    SIM_KERNEL_KINDS = 4
};

/* sim_profile: on != 0 makes every later kernel launch of h (outside a graph
 * capture) record a CUDA event pair around itself on its own stream, so each
 * kernel's device duration is measured where it runs.  At most 65536 pairs
 * are kept between resets of sim_kernel_times. */
int sim_profile(sim_handle *h, int32_t on);

/* sim_kernel_times: ms (HOST double[SIM_KERNEL_KINDS], nullable) receives the
 * summed device milliseconds of the profiled launches per kind (waits for
 * them); launches (HOST int64[SIM_KERNEL_KINDS], nullable) the number of
 * kernels h launched per kind, profiled or not, graph launches included.
 * reset != 0 clears both afterwards.  SIM_ERR_SIZE if event pairs ran out
 * (the times then cover only the first 65536 launches). */
int sim_kernel_times(sim_handle *h, double *ms, int64_t *launches, int32_t reset);

/* Buffers of a captured reset + rollout (+ adjoint); all DEVICE pointers with
 * the layouts of sim_reset, sim_rollout and sim_backward.  g_r == NULL
 * captures no adjoint. */
typedef struct sim_graph_io {
    const float *state0; /* [NM][D]; NULL: pool entry 0 */
    const float *actions;
    float *r_ctrl;
    int8_t *r_goal;
    uint8_t *done;
    float *depth, *lidar;
    const float *g_r, *g_depth, *g_lidar, *g_sT;
    float *g_a, *g_s0;
} sim_graph_io;

typedef struct sim_graph sim_graph;

/* sim_graph_create: captures sim_reset + sim_rollout (+ sim_backward) of h
 * with the buffers of io (HOST struct) into one CUDA graph (a memcpy, memsets
 * and 2 or 4 kernels), launched by sim_graph_launch without any host work
 * per kernel.  Nothing runs during creation.  The pointers in io are baked
 * in: they stay valid while the graph is used.  A later sim_set_scene,
 * sim_set_pool or sim_set_env_params on h makes the graph refuse to launch
 * (SIM_ERR_NOT_READY); sim_destroy(h) does too (the sim_graph object itself
 * stays owned by the caller).  Errors: those of the captured calls. */
int sim_graph_create(sim_handle *h, const sim_graph_io *io, sim_graph **out);

/* sim_graph_launch: one reset + rollout (+ adjoint) on stream.  Afterwards h
 * holds that rollout, as if the captured calls had been made. */
int sim_graph_launch(sim_graph *g, sim_stream_t stream);

/* sim_graph_kernels: number of kernel nodes in the graph (HOST out). */
int sim_graph_kernels(const sim_graph *g, int32_t *kernels);

/* sim_graph_destroy: waits for h's last stream and frees the graph; NULL-safe. */
int sim_graph_destroy(sim_graph *g);

#ifdef __cplusplus
}
#endif

#endif /* DIFFSIM_H */
