/*
 * diffsim_oracle.c -- plain FP64 CPU oracle of the batched, differentiable
 * quadrotor environment step of DiffAero (arXiv 2509.10247).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library) never links, imports or calls it, and it shares no code with it.
 *
 * What it computes, in the paper's order and notation:
 *   - continuous point-mass dynamics (Sec. III-A, Eq. 3) and full rigid-body
 *     quadrotor dynamics (Sec. III-A, Eq. 1) with the body-rate part of the
 *     geometric controller, integrated by explicit Euler with every right-hand
 *     side taken at time t (the paper gives only the continuous equations);
 *   - point-mass attitude from the thrust direction and the horizontal
 *     projection of an exponential moving average of velocity (Sec. III-B);
 *   - depth camera and LiDAR by ray casting against analytic spheres,
 *     axis-aligned boxes, vertical capped cylinders and racing-gate frames
 *     (Sec. III-B: one ray-casting function per primitive shape), brute force
 *     over every primitive, no field-of-view culling (culling only skips
 *     primitives no ray can hit);
 *   - collisions, the dense differentiable reward R_ctrl and the sparse
 *     reward R_goal (Sec. III-C, III-D, III-E), termination and reset;
 *   - the reverse-mode adjoint of the whole rollout, i.e. the chain rule of
 *     Eq. 5 taken one step at a time, written by hand.
 * All arithmetic is double precision.  Where the paper is silent the reading
 * taken is the one listed in the design notes (e.g. thrust along +z_B in a
 * z-up world; lambda = 1/tau; z-depth output clamped at the camera range).
 *
 * Layouts (row-major, last index fastest):
 *   state  [NM][D], D = 12 (point mass: p, v, a, ema_v) or 13 (rigid: p,
 *          q=(w,x,y,z), v, omega); actions [T][NM][A], A = 3 or 4;
 *   spheres [K][4] = (cx, cy, cz, r); boxes [K][6] = (min xyz, max xyz);
 *   cylinders [K][5] = (cx, cy, r, zmin, zmax), axis along world z;
 *   gates [K][7] = (cx, cy, cz, yaw, w, b, hd): a square frame whose opening
 *   has half-width w, border width b and half-depth hd along its normal
 *   (cos yaw, sin yaw, 0); per-map CSR offsets; env_map [N]; targets [NM][3];
 *   pool [P][NM][D].  Primitive ids within a map: spheres 0..ns-1, boxes
 *   ns..ns+nb-1, cylinders from ns+nb, gates from ns+nb+nc.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_PM 0
#define OC_RIGID 1
#define OC_PMD 2    /* discrete point mass, Eq. 4 */
#define OC_SIMPLE 3 /* simplified quadrotor, Eq. 2 */
#define OC_INF HUGE_VAL

/* Ambiguity margins used to flag rays and steps where an FP32 evaluation may
 * legitimately take another discrete branch than FP64 (see the design notes). */
#define AMB_DISC 1e-5   /* sphere grazing: |b^2 - C| < AMB_DISC * max(b^2, 1)  */
#define AMB_SLAB 1e-5   /* box grazing: |t_far - t_near| < AMB_SLAB (m)        */
#define AMB_INSIDE 1e-5 /* origin within this distance of a primitive surface  */
#define AMB_GAP 1e-4    /* second-nearest hit within this distance (m)         */
#define AMB_RANGE 1e-4  /* hit within this distance of the range clamp (m)     */
#define AMB_GRAZE 0.05  /* |n . d| below this: ill-conditioned gradient       */
#define AMB_EDGE 1e-4   /* two slab entry times within this (relative)        */
#define AMB_STEP 1e-5   /* thresholds of collision / success / bounds (m)     */
#define COND_DIR 3e-7   /* FP32 error of a rotated unit ray direction          */
#define COND_ORG 1e-6   /* FP32 error of an origin-relative coordinate (m)    */
#define COND_MAX 5e-5   /* half of the 1e-4 m depth tolerance                 */
#define DRIFT_POS 1e-5  /* position drift of an FP32 rollout vs FP64 (m)      */

typedef struct {
    int32_t model, n_env, n_agent, horizon;
    double dt, gravity;
    /* point mass (Eq. 3) */
    double lam, drag, act_scale, ema_alpha;
    /* rigid body (Eq. 1) */
    double mass, inertia[3], k_rate[3], drag_body[3], rate_scale[3];
    /* depth camera; cam_w == 0 disables it.  Angles in radians. */
    int32_t cam_w, cam_h;
    double cam_hfov, cam_range;
    /* lidar; lid_ch == 0 disables it */
    int32_t lid_ch, lid_az;
    double lid_elev_lo, lid_elev_hi, lid_range;
    /* task and reward */
    int32_t pos_sq;
    double w_pos, w_obs, d_safe, w_act, w_agent, d_agent, success_radius, r_quad;
    double bound_lo[3], bound_hi[3];
    int32_t terminate, pool_size;
    /* task 0: reach targets / avoid obstacles; 1: racing through the map's
     * gates in order (Sec. III-C), progress reward as in the design notes */
    int32_t task;
    /* IMU noise (Sec. III-B): white-noise standard deviation of the specific
     * force (m/s^2) and angular rate (rad/s) samples, and the standard
     * deviations per sqrt(s) of their bias random walks */
    double imu_noise[2], imu_walk[2];
} oc_config;

typedef struct {
    const double *spheres;
    const int32_t *sph_off;
    const double *boxes;
    const int32_t *box_off;
    const double *cylinders; /* NULL: none */
    const int32_t *cyl_off;
    const double *gates;     /* NULL: none */
    const int32_t *gate_off;
    const int32_t *env_map;
    int32_t n_maps;
    const double *targets;
    const double *pool;
    const double *drag_env; /* [N] or NULL */
    const double *lam_env;  /* [N] or NULL */
} oc_scene;

/* Per-rollout task and IMU state, any pointer NULL when unused. */
typedef struct {
    int32_t *gate_k;         /* [NM] racing: each agent's next gate, read and advanced */
    int32_t *gate_tape;      /* [T][NM] out: the gate each agent targets during step t */
    double *imu;             /* [T][NM][6] out: specific force, angular rate (body frame) */
    const double *imu_noise; /* [T][NM][12] standard normal samples: 6 white, 6 bias steps */
    double *imu_bias;        /* [NM][6] bias, read and advanced (with imu_noise) */
} oc_extra;

/* ------------------------------------------------------------------ utils */
int oc_state_dim(int model) { return model == OC_RIGID ? 13 : (model == OC_SIMPLE ? 15 : 12); }
int oc_action_dim(int model) { return (model == OC_RIGID || model == OC_SIMPLE) ? 4 : 3; }

static double clamp1(double x) { return x < -1.0 ? -1.0 : (x > 1.0 ? 1.0 : x); }
static double dclamp1(double x) { return (x >= -1.0 && x <= 1.0) ? 1.0 : 0.0; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }
static void cross3(const double *a, const double *b, double *o)
{
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double relu(double x) { return x > 0.0 ? x : 0.0; }

/* R(q): rotation body -> world of the Hamilton unit quaternion q = (w, x, y, z),
 * row-major R[3*i + j]. */
void oc_quat_to_rot(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* cotangent of q from the cotangent of R(q) (the entries' partial derivatives
 * of the polynomial map above). */
static void quat_to_rot_vjp(const double *q, const double *gR, double *gq)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    const double dw[9] = {0, -z, y, z, 0, -x, -y, x, 0};
    const double dx[9] = {0, y, z, y, -2 * x, -w, z, w, -2 * x};
    const double dy[9] = {-2 * y, x, w, x, 0, z, -w, z, -2 * y};
    const double dz[9] = {-2 * z, -w, x, w, -2 * z, y, x, y, 0};
    double s[4] = {0, 0, 0, 0};
    for (int k = 0; k < 9; ++k) {
        s[0] += 2 * dw[k] * gR[k];
        s[1] += 2 * dx[k] * gR[k];
        s[2] += 2 * dy[k] * gR[k];
        s[3] += 2 * dz[k] * gR[k];
    }
    for (int k = 0; k < 4; ++k) gq[k] += s[k];
}

/* Hamilton product a (x) b */
static void quat_mul(const double *a, const double *b, double *o)
{
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

/* ------------------------------------------------------ dynamics (Sec. III-A) */

/* Continuous point mass, Eq. 3: p' = v, v' = a + g - d v, a' = lambda (u - a),
 * one explicit-Euler step of length dt; u = act_scale * clip(action, -1, 1) is
 * the world-frame acceleration command.  The EMA of velocity used by the
 * point-mass attitude (Sec. III-B) is advanced from the new velocity. */
void oc_pm_step(const oc_config *c, double drag, double lam, const double *s,
                const double *act, double *o)
{
    const double g[3] = {0.0, 0.0, -c->gravity};
    double u[3], n[12];
    for (int i = 0; i < 3; ++i) u[i] = c->act_scale * clamp1(act[i]);
    for (int i = 0; i < 3; ++i) {
        double p = s[i], v = s[3 + i], a = s[6 + i], e = s[9 + i];
        n[i] = p + c->dt * v;
        n[3 + i] = v + c->dt * (a + g[i] - drag * v);
        n[6 + i] = a + c->dt * lam * (u[i] - a);
        n[9 + i] = (1.0 - c->ema_alpha) * e + c->ema_alpha * n[3 + i];
    }
    memcpy(o, n, sizeof(n));
}

/* Full quadrotor, Eq. 1: p' = v, v' = g + c z_B - R D R^T v (thrust along +z_B,
 * c = T/m), q' = 1/2 q (x) [0, omega], omega' = J^-1 (tau - omega x J omega).
 * The controller takes a thrust command T = m g (1 + clip(a0)) and a body-rate
 * command omega_c = rate_scale * clip(a1..3); its torque is the body-rate part
 * of the geometric controller, tau = J K (omega_c - omega) + omega x J omega.
 * One explicit-Euler step; the quaternion is renormalised after the update. */
void oc_rb_step(const oc_config *c, const double *s, const double *act, double *o)
{
    const double *p = s, *q = s + 3, *v = s + 7, *w = s + 10;
    const double *J = c->inertia;
    double T = c->mass * c->gravity * (1.0 + clamp1(act[0]));
    double wc[3], Jw[3], gy[3], tau[3], wd[3], R[9], vb[3], dw[3], vd[3];
    for (int i = 0; i < 3; ++i) wc[i] = c->rate_scale[i] * clamp1(act[1 + i]);
    for (int i = 0; i < 3; ++i) Jw[i] = J[i] * w[i];
    cross3(w, Jw, gy);
    for (int i = 0; i < 3; ++i) tau[i] = J[i] * c->k_rate[i] * (wc[i] - w[i]) + gy[i];
    for (int i = 0; i < 3; ++i) wd[i] = (tau[i] - gy[i]) / J[i];
    oc_quat_to_rot(q, R);
    for (int j = 0; j < 3; ++j) vb[j] = R[0 + j] * v[0] + R[3 + j] * v[1] + R[6 + j] * v[2];
    for (int j = 0; j < 3; ++j) vb[j] *= c->drag_body[j];
    for (int i = 0; i < 3; ++i) dw[i] = R[3 * i] * vb[0] + R[3 * i + 1] * vb[1] + R[3 * i + 2] * vb[2];
    const double g[3] = {0.0, 0.0, -c->gravity};
    for (int i = 0; i < 3; ++i) vd[i] = g[i] + (T / c->mass) * R[3 * i + 2] - dw[i];
    double qw[4] = {0.0, w[0], w[1], w[2]}, qd[4];
    quat_mul(q, qw, qd);
    double n[13], qt[4];
    for (int i = 0; i < 3; ++i) n[i] = p[i] + c->dt * v[i];
    for (int k = 0; k < 4; ++k) qt[k] = q[k] + c->dt * 0.5 * qd[k];
    double nq = sqrt(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
    for (int k = 0; k < 4; ++k) n[3 + k] = qt[k] / nq;
    for (int i = 0; i < 3; ++i) n[7 + i] = v[i] + c->dt * vd[i];
    for (int i = 0; i < 3; ++i) n[10 + i] = w[i] + c->dt * wd[i];
    memcpy(o, n, sizeof(n));
}

/* Discrete point mass, Eq. 4: p_{t+1} = p_t + v_t dt + 1/2 w_t dt^2,
 * v_{t+1} = v_t + 1/2 (w_t + w_{t+1}) dt, with w the total acceleration.  The
 * state's acceleration slot carries the thrust acceleration u_t of the
 * command in force (w_t = u_t + g); the step's action is the next command,
 * u_{t+1} = act_scale * clip(action), so the half-step average of Eq. 4 needs
 * no look-ahead.  The velocity EMA (attitude, Sec. III-B) follows v_{t+1}. */
void oc_pmd_step(const oc_config *c, const double *s, const double *act, double *o)
{
    const double g[3] = {0.0, 0.0, -c->gravity};
    const double dt = c->dt;
    double n[12];
    for (int i = 0; i < 3; ++i) {
        double p = s[i], v = s[3 + i], u = s[6 + i], e = s[9 + i];
        double u1 = c->act_scale * clamp1(act[i]);
        n[i] = p + v * dt + 0.5 * (u + g[i]) * dt * dt;
        n[3 + i] = v + 0.5 * ((u + g[i]) + (u1 + g[i])) * dt;
        n[6 + i] = u1;
        n[9 + i] = (1.0 - c->ema_alpha) * e + c->ema_alpha * n[3 + i];
    }
    memcpy(o, n, sizeof(n));
}

/* Simplified quadrotor, Eq. 2: p' = v, v' = R c e3 + g, R' = R [omega]_x, with
 * the collective thrust acceleration c = g (1 + clip(a0)) (hover at a0 = 0)
 * and body rates omega = rate_scale * clip(a1..3) taken directly as inputs.
 * State (p, v, R) with R row-major, body -> world.  One explicit-Euler step,
 * then the rotation is re-orthonormalised by Gram-Schmidt on its columns
 * (x normalised, y made orthogonal to x and normalised, z = x cross y). */
static void simple_pre(const oc_config *c, const double *s, const double *act, double *Rt, double *w,
                       double *cth)
{
    const double *R = s + 6;
    *cth = c->gravity * (1.0 + clamp1(act[0]));
    for (int i = 0; i < 3; ++i) w[i] = c->rate_scale[i] * clamp1(act[1 + i]);
    /* Rt = R + dt R [w]_x;  column j of R [w]_x is R (w x e_j) */
    const double W[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * W[3 * k + j];
            Rt[3 * i + j] = R[3 * i + j] + c->dt * acc;
        }
}

static void gram_schmidt(const double *Rt, double *Ro)
{
    double u0[3] = {Rt[0], Rt[3], Rt[6]}, u1[3] = {Rt[1], Rt[4], Rt[7]};
    double n0 = norm3(u0), x[3], wv[3], y[3], z[3];
    for (int i = 0; i < 3; ++i) x[i] = u0[i] / n0;
    double sx = dot3(x, u1);
    for (int i = 0; i < 3; ++i) wv[i] = u1[i] - sx * x[i];
    double n1 = norm3(wv);
    for (int i = 0; i < 3; ++i) y[i] = wv[i] / n1;
    cross3(x, y, z);
    for (int i = 0; i < 3; ++i) { Ro[3 * i] = x[i]; Ro[3 * i + 1] = y[i]; Ro[3 * i + 2] = z[i]; }
}

void oc_simple_step(const oc_config *c, const double *s, const double *act, double *o)
{
    const double *p = s, *v = s + 3, *R = s + 6;
    double Rt[9], w[3], cth, n[15];
    simple_pre(c, s, act, Rt, w, &cth);
    const double g[3] = {0.0, 0.0, -c->gravity};
    for (int i = 0; i < 3; ++i) {
        n[i] = p[i] + c->dt * v[i];
        n[3 + i] = v[i] + c->dt * (R[3 * i + 2] * cth + g[i]);
    }
    gram_schmidt(Rt, n + 6);
    memcpy(o, n, sizeof(n));
}

/* ------------------------------------------------------ attitude (Sec. III-B) */

/* Sensor pose of one agent: origin = position, R = body->world rotation.
 * Rigid body: R(q).  Point mass: z_B along the thrust acceleration a; x_B is
 * the horizontal projection of the velocity EMA, made orthogonal to z_B;
 * y_B = z_B x x_B.  Degenerate cases: |a| < 1e-6 -> z_B = +z; horizontal
 * heading (after orthogonalisation) shorter than 1e-6 -> world +x is used as
 * heading instead, then world +y.  Returns a flag word: bit 0 = |a| fallback,
 * bit 1 = heading fallback, bit 2 = a decision within 1e-3 relative of its
 * threshold (ambiguous in FP32). */
int oc_pose(const oc_config *c, const double *s, double *o, double *R)
{
    o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
    if (c->model == OC_RIGID) {
        oc_quat_to_rot(s + 3, R);
        return 0;
    }
    if (c->model == OC_SIMPLE) {
        memcpy(R, s + 6, 9 * sizeof(double));
        return 0;
    }
    int flags = 0;
    const double *a = s + 6, *e = s + 9;
    double z[3], x[3], y[3];
    double na = norm3(a);
    if (na < 1e-6) { z[0] = 0; z[1] = 0; z[2] = 1; flags |= 1; }
    else { z[0] = a[0] / na; z[1] = a[1] / na; z[2] = a[2] / na; }
    if (fabs(na - 1e-6) < 1e-9) flags |= 4;
    double h[3] = {e[0], e[1], 0.0}, hp[3];
    double hz = dot3(h, z);
    for (int i = 0; i < 3; ++i) hp[i] = h[i] - hz * z[i];
    double nh = norm3(hp);
    if (fabs(nh - 1e-6) < 1e-9) flags |= 4;
    if (nh < 1e-6) {
        flags |= 2;
        double hx[3] = {1, 0, 0};
        hz = dot3(hx, z);
        for (int i = 0; i < 3; ++i) hp[i] = hx[i] - hz * z[i];
        nh = norm3(hp);
        if (nh < 1e-6) {
            double hy[3] = {0, 1, 0};
            hz = dot3(hy, z);
            for (int i = 0; i < 3; ++i) hp[i] = hy[i] - hz * z[i];
            nh = norm3(hp);
        }
    }
    for (int i = 0; i < 3; ++i) x[i] = hp[i] / nh;
    cross3(z, x, y);
    for (int i = 0; i < 3; ++i) { R[3 * i] = x[i]; R[3 * i + 1] = y[i]; R[3 * i + 2] = z[i]; }
    return flags;
}

/* Conditioning of the sensor attitude at state s (Sec. III-B): the factor by
 * which FP32 rounding of the state (and of the arithmetic) is amplified in
 * the body axes, relative to a well-conditioned rotation.  Rigid body and
 * simplified quadrotor: 1 (the rotation is the state).  Point mass: x_B is
 * the heading vector h with its z_B component removed, normalised; rounding h
 * and z_B moves that difference by ~eps |h|, so x_B turns by ~eps |h| /
 * |h - (h.z_B) z_B|: the factor is |h| / |h_perp| (>= 1), of the vector the
 * rule actually uses (the heading, else the world-axis fallback). */
static double pose_kappa(const oc_config *c, const double *s)
{
    if (c->model != OC_PM && c->model != OC_PMD) return 1.0;
    const double *a = s + 6, *e = s + 9;
    double z[3] = {0.0, 0.0, 1.0};
    double na = norm3(a);
    if (na >= 1e-6) { z[0] = a[0] / na; z[1] = a[1] / na; z[2] = a[2] / na; }
    double cand[3][3] = {{e[0], e[1], 0.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}};
    for (int k = 0; k < 3; ++k) {
        const double *h = cand[k];
        double hz = dot3(h, z), hp[3];
        for (int i = 0; i < 3; ++i) hp[i] = h[i] - hz * z[i];
        double nh = norm3(hp);
        if (nh >= 1e-6 || k == 2) {
            double r = norm3(h) / (nh > 0.0 ? nh : 1e-300);
            return r > 1.0 ? r : 1.0;
        }
    }
    return 1.0;
}

/* ------------------------------------------------------- sensors (Sec. III-B) */

/* Depth-camera rays in the body frame: pinhole looking along +x_B, image
 * column i to the right (-y_B), row j downwards (-z_B), pixel centres,
 * horizontal field of view hfov and square pixels.  Ray index j * W + i.
 * dir [R][3] unit vectors; fac [R] = cos of the angle to the optical axis,
 * which turns ray distance into z-depth. */
void oc_cam_dirs(const oc_config *c, double *dir, double *fac)
{
    int W = c->cam_w, H = c->cam_h;
    double th = tan(0.5 * c->cam_hfov), tv = th * (double)H / (double)W;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double u = (2.0 * (i + 0.5) / W - 1.0) * th;
            double v = (2.0 * (j + 0.5) / H - 1.0) * tv;
            double d[3] = {1.0, -u, -v};
            double n = norm3(d);
            int r = j * W + i;
            for (int k = 0; k < 3; ++k) dir[3 * r + k] = d[k] / n;
            fac[r] = 1.0 / n;
        }
}

/* LiDAR rays in the body frame: C channels at elevations evenly spaced over
 * [elev_lo, elev_hi] (inclusive), Az azimuths k * 360/Az degrees from +x_B
 * towards +y_B.  Ray index ch * Az + k. */
void oc_lidar_dirs(const oc_config *c, double *dir)
{
    int C = c->lid_ch, Az = c->lid_az;
    for (int ch = 0; ch < C; ++ch) {
        double el = C > 1 ? c->lid_elev_lo + ch * (c->lid_elev_hi - c->lid_elev_lo) / (C - 1)
                          : 0.5 * (c->lid_elev_lo + c->lid_elev_hi);
        for (int k = 0; k < Az; ++k) {
            double az = 2.0 * M_PI * k / Az;
            int r = ch * Az + k;
            dir[3 * r + 0] = cos(el) * cos(az);
            dir[3 * r + 1] = cos(el) * sin(az);
            dir[3 * r + 2] = sin(el);
        }
    }
}

/* Ray vs sphere: smallest t >= 0 with |o + t d - c| = r, |d| = 1; 0 when the
 * origin is inside or on the sphere; +inf on a miss. */
double oc_ray_sphere(const double *o, const double *d, const double *sp)
{
    double oc[3] = {sp[0] - o[0], sp[1] - o[1], sp[2] - o[2]};
    double C = dot3(oc, oc) - sp[3] * sp[3];
    if (C <= 0.0) return 0.0;
    double b = dot3(d, oc);
    double disc = b * b - C;
    if (disc < 0.0 || b <= 0.0) return OC_INF;
    return b - sqrt(disc);
}

/* Ray vs axis-aligned box by slabs: entry t_n = max_i min(t1_i, t2_i), exit
 * t_f = min_i max(t1_i, t2_i); hit iff t_n <= t_f and t_f >= 0; 0 when the
 * origin is inside.  A direction component of exactly 0 keeps the slab only
 * if the origin lies between its planes.  *axis receives the entry axis. */
double oc_ray_box(const double *o, const double *d, const double *bx, int *axis)
{
    double tn = -OC_INF, tf = OC_INF;
    int ax = -1;
    for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0) {
            if (o[i] < bx[i] || o[i] > bx[3 + i]) return OC_INF;
            continue;
        }
        double t1 = (bx[i] - o[i]) / d[i], t2 = (bx[3 + i] - o[i]) / d[i];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tn) { tn = lo; ax = i; }
        if (hi < tf) tf = hi;
    }
    if (axis) *axis = ax;
    if (tn > tf || tf < 0.0) return OC_INF;
    return tn > 0.0 ? tn : 0.0;
}

/* Signed distance from a point to a sphere and to a box (exact Euclidean). */
double oc_sdf_sphere(const double *p, const double *sp)
{
    double d[3] = {p[0] - sp[0], p[1] - sp[1], p[2] - sp[2]};
    return norm3(d) - sp[3];
}

double oc_sdf_box(const double *p, const double *bx)
{
    double q[3], out = 0.0, in = -OC_INF;
    for (int i = 0; i < 3; ++i) {
        double ctr = 0.5 * (bx[i] + bx[3 + i]), half = 0.5 * (bx[3 + i] - bx[i]);
        q[i] = fabs(p[i] - ctr) - half;
        out += relu(q[i]) * relu(q[i]);
        if (q[i] > in) in = q[i];
    }
    return sqrt(out) + (in < 0.0 ? in : 0.0);
}

/* gradient of the box SDF w.r.t. the point */
static void sdf_box_grad(const double *p, const double *bx, double *gp)
{
    double q[3], sg[3], out = 0.0;
    int am = 0;
    for (int i = 0; i < 3; ++i) {
        double ctr = 0.5 * (bx[i] + bx[3 + i]), half = 0.5 * (bx[3 + i] - bx[i]);
        sg[i] = p[i] - ctr >= 0.0 ? 1.0 : -1.0;
        q[i] = fabs(p[i] - ctr) - half;
        out += relu(q[i]) * relu(q[i]);
        if (q[i] > q[am]) am = i;
    }
    if (out > 0.0) {
        double n = sqrt(out);
        for (int i = 0; i < 3; ++i) gp[i] = relu(q[i]) * sg[i] / n;
    } else {
        for (int i = 0; i < 3; ++i) gp[i] = (i == am) ? sg[i] : 0.0;
    }
}

/* Ray vs vertical capped cylinder cy = (cx, cy, r, zmin, zmax): the solid is
 * the intersection of the infinite cylinder (x - cx)^2 + (y - cy)^2 <= r^2
 * (a quadratic in the ray parameter) and the slab zmin <= z <= zmax.  Entry =
 * the later of the two entries, exit = the earlier exit; hit iff entry <=
 * exit and exit >= 0; 0 when the origin is inside.  A ray parallel to the
 * axis keeps the quadratic interval only from inside the infinite cylinder,
 * a horizontal ray the slab only from between its planes.  *face receives 0
 * for an entry through the side, 1 through a cap. */
double oc_ray_cylinder(const double *o, const double *d, const double *cy, int *face)
{
    double ex = o[0] - cy[0], ey = o[1] - cy[1];
    double a = d[0] * d[0] + d[1] * d[1];
    double b = d[0] * ex + d[1] * ey;
    double cc = ex * ex + ey * ey - cy[2] * cy[2];
    double s0, s1, z0, z1;
    if (a == 0.0) {
        if (cc > 0.0) return OC_INF;
        s0 = -OC_INF; s1 = OC_INF;
    } else {
        double disc = b * b - a * cc;
        if (disc < 0.0) return OC_INF;
        double sq = sqrt(disc);
        s0 = (-b - sq) / a; s1 = (-b + sq) / a;
    }
    if (d[2] == 0.0) {
        if (o[2] < cy[3] || o[2] > cy[4]) return OC_INF;
        z0 = -OC_INF; z1 = OC_INF;
    } else {
        double t1 = (cy[3] - o[2]) / d[2], t2 = (cy[4] - o[2]) / d[2];
        z0 = t1 < t2 ? t1 : t2; z1 = t1 < t2 ? t2 : t1;
    }
    double tn = s0 > z0 ? s0 : z0, tf = s1 < z1 ? s1 : z1;
    if (face) *face = s0 >= z0 ? 0 : 1;
    if (tn > tf || tf < 0.0) return OC_INF;
    return tn > 0.0 ? tn : 0.0;
}

/* Signed distance to the capped cylinder: radial excess q_r = rho - r and
 * axial excess q_z = |z - zc| - hz combine like a 2D box. */
double oc_sdf_cylinder(const double *p, const double *cy)
{
    double rho = hypot(p[0] - cy[0], p[1] - cy[1]);
    double zc = 0.5 * (cy[3] + cy[4]), hz = 0.5 * (cy[4] - cy[3]);
    double qr = rho - cy[2], qz = fabs(p[2] - zc) - hz;
    double in = qr > qz ? qr : qz;
    return sqrt(relu(qr) * relu(qr) + relu(qz) * relu(qz)) + (in < 0.0 ? in : 0.0);
}

static void sdf_cylinder_grad(const double *p, const double *cy, double *gp)
{
    double ex = p[0] - cy[0], ey = p[1] - cy[1];
    double rho = hypot(ex, ey);
    double zc = 0.5 * (cy[3] + cy[4]), hz = 0.5 * (cy[4] - cy[3]);
    double qr = rho - cy[2], qz = fabs(p[2] - zc) - hz;
    double ur[2] = {rho > 0.0 ? ex / rho : 0.0, rho > 0.0 ? ey / rho : 0.0};
    double sz = p[2] - zc >= 0.0 ? 1.0 : -1.0;
    double out = sqrt(relu(qr) * relu(qr) + relu(qz) * relu(qz));
    if (out > 0.0) {
        gp[0] = relu(qr) * ur[0] / out;
        gp[1] = relu(qr) * ur[1] / out;
        gp[2] = relu(qz) * sz / out;
    } else if (qr >= qz) {
        gp[0] = ur[0]; gp[1] = ur[1]; gp[2] = 0.0;
    } else {
        gp[0] = 0.0; gp[1] = 0.0; gp[2] = sz;
    }
}

/* Racing gate g = (cx, cy, cz, yaw, w, b, hd).  Its frame: normal
 * n = (cos yaw, sin yaw, 0), lateral l = (-sin yaw, cos yaw, 0), up z.  Local
 * coordinates of a point x: u = (n.(x - c), l.(x - c), z - cz).  The solid is
 * the box |u_n| <= hd, |u_l| <= w + b, |u_z| <= w + b without the open
 * square |u_l| < w, |u_z| < w (all u_n): a frame of four bars. */
static void gate_axes(const double *g, double *n, double *l)
{
    double cs = cos(g[3]), sn = sin(g[3]);
    n[0] = cs; n[1] = sn; n[2] = 0.0;
    l[0] = -sn; l[1] = cs; l[2] = 0.0;
}

static void gate_local(const double *g, const double *x, int is_dir, double *u)
{
    double n[3], l[3], r[3];
    gate_axes(g, n, l);
    for (int i = 0; i < 3; ++i) r[i] = x[i] - (is_dir ? 0.0 : g[i]);
    u[0] = dot3(n, r); u[1] = dot3(l, r); u[2] = r[2];
}

static void gate_world(const double *g, const double *u, double *x)
{
    double n[3], l[3];
    gate_axes(g, n, l);
    for (int i = 0; i < 3; ++i) x[i] = u[0] * n[i] + u[1] * l[i] + (i == 2 ? u[2] : 0.0);
}

/* Ray vs gate frame.  The ray meets the outer box over [t_n, t_f] (slabs in
 * local coordinates) and the open square prism over (i_n, i_f) (slabs in u_l
 * and u_z only).  The first solid point at or after max(t_n, 0) is that point
 * itself unless it lies strictly inside the prism; then it is where the ray
 * leaves the prism, i_f, if that is still inside the outer box.  0 when the
 * origin is in the solid.  *axis: 0..2 = outer face entered (u_n, u_l, u_z),
 * 3 / 4 = inner wall met (u_l / u_z), -1 at t = 0. */
double oc_ray_gate(const double *o, const double *d, const double *g, int *axis)
{
    double uo[3], ud[3];
    gate_local(g, o, 0, uo);
    gate_local(g, d, 1, ud);
    double W = g[4] + g[5], half[3] = {g[6], W, W};
    double tn = -OC_INF, tf = OC_INF, in = -OC_INF, inf_ = OC_INF;
    int ax = -1, bx = -1, open = 1;
    for (int i = 0; i < 3; ++i) {
        if (ud[i] == 0.0) {
            if (fabs(uo[i]) > half[i]) return OC_INF;
            continue;
        }
        double t1 = (-half[i] - uo[i]) / ud[i], t2 = (half[i] - uo[i]) / ud[i];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tn) { tn = lo; ax = i; }
        if (hi < tf) tf = hi;
    }
    if (tn > tf || tf < 0.0) return OC_INF;
    for (int i = 1; i < 3; ++i) {
        if (ud[i] == 0.0) {
            if (fabs(uo[i]) >= g[4]) open = 0;
            continue;
        }
        double t1 = (-g[4] - uo[i]) / ud[i], t2 = (g[4] - uo[i]) / ud[i];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > in) in = lo;
        if (hi < inf_) { inf_ = hi; bx = i; }
    }
    if (in >= inf_) open = 0;
    double ta = tn > 0.0 ? tn : 0.0;
    if (!open || ta <= in || ta >= inf_) {
        if (axis) *axis = tn > 0.0 ? ax : -1;
        return ta;
    }
    if (inf_ <= tf) {
        if (axis) *axis = 2 + bx;
        return inf_;
    }
    return OC_INF;
}

/* The gate's four bars as boxes in local coordinates (min u, max u):
 * top and bottom span the full outer width, left and right the opening's
 * height, so the bars tile the frame without overlap. */
static void gate_bar(const double *g, int k, double *bx)
{
    double w = g[4], b = g[5], hd = g[6], W = w + b, m = w + 0.5 * b;
    double cl = 0.0, cz = 0.0, hl, hz;
    if (k < 2) { cz = k == 0 ? m : -m; hl = W; hz = 0.5 * b; }
    else { cl = k == 2 ? -m : m; hl = 0.5 * b; hz = w; }
    bx[0] = -hd; bx[1] = cl - hl; bx[2] = cz - hz;
    bx[3] = hd; bx[4] = cl + hl; bx[5] = cz + hz;
}

/* Signed distance to the gate: the minimum over its four bars (exact outside
 * the frame, negative inside it).  *bar receives the arg-min bar. */
double oc_sdf_gate(const double *p, const double *g, int *bar)
{
    double u[3], best = OC_INF;
    int bi = 0;
    gate_local(g, p, 0, u);
    for (int k = 0; k < 4; ++k) {
        double bx[6];
        gate_bar(g, k, bx);
        double s = oc_sdf_box(u, bx);
        if (s < best) { best = s; bi = k; }
    }
    if (bar) *bar = bi;
    return best;
}

static void sdf_gate_grad(const double *p, const double *g, double *gp)
{
    double u[3], bx[6], gu[3];
    int k;
    oc_sdf_gate(p, g, &k);
    gate_local(g, p, 0, u);
    gate_bar(g, k, bx);
    sdf_box_grad(u, bx, gu);
    gate_world(g, gu, gp);
}

/* ------------------------------------------------------------ maps */

/* The primitives of one map, by kind. */
typedef struct {
    const double *sph, *box, *cyl, *gate;
    int ns, nb, nc, ng;
} map_t;

static int map_count(const map_t *m) { return m->ns + m->nb + m->nc + m->ng; }

/* Ray parameter of the first hit of primitive id (aux: box entry axis,
 * cylinder face or gate axis). */
static double prim_ray(const map_t *m, int id, const double *o, const double *d, int *aux)
{
    *aux = -1;
    if (id < m->ns) return oc_ray_sphere(o, d, m->sph + 4 * id);
    id -= m->ns;
    if (id < m->nb) return oc_ray_box(o, d, m->box + 6 * id, aux);
    id -= m->nb;
    if (id < m->nc) return oc_ray_cylinder(o, d, m->cyl + 5 * id, aux);
    return oc_ray_gate(o, d, m->gate + 7 * (id - m->nc), aux);
}

/* Outward unit normal of primitive id at the hit o + t d (t > 0); false when
 * the hit has no face (aux -1). */
static int prim_normal(const map_t *m, int id, const double *o, const double *d, double t, int aux, double *n)
{
    for (int i = 0; i < 3; ++i) n[i] = 0.0;
    if (id < m->ns) {
        const double *sp = m->sph + 4 * id;
        for (int i = 0; i < 3; ++i) n[i] = (o[i] + t * d[i] - sp[i]) / sp[3];
        return 1;
    }
    id -= m->ns;
    if (aux < 0) return 0;
    if (id < m->nb) {
        n[aux] = d[aux] > 0.0 ? -1.0 : 1.0;
        return 1;
    }
    id -= m->nb;
    if (id < m->nc) {
        const double *cy = m->cyl + 5 * id;
        if (aux == 1) { n[2] = d[2] > 0.0 ? -1.0 : 1.0; return 1; }
        n[0] = (o[0] + t * d[0] - cy[0]) / cy[2];
        n[1] = (o[1] + t * d[1] - cy[1]) / cy[2];
        return 1;
    }
    const double *g = m->gate + 7 * (id - m->nc);
    double ud[3], un[3] = {0.0, 0.0, 0.0};
    gate_local(g, d, 1, ud);
    int k = aux < 3 ? aux : aux - 2;
    un[k] = ud[k] > 0.0 ? -1.0 : 1.0;
    gate_world(g, un, n);
    return 1;
}

static double prim_sdf(const map_t *m, int id, const double *p)
{
    if (id < m->ns) return oc_sdf_sphere(p, m->sph + 4 * id);
    id -= m->ns;
    if (id < m->nb) return oc_sdf_box(p, m->box + 6 * id);
    id -= m->nb;
    if (id < m->nc) return oc_sdf_cylinder(p, m->cyl + 5 * id);
    return oc_sdf_gate(p, m->gate + 7 * (id - m->nc), NULL);
}

/* Slab-type decisions of primitive id that are near their thresholds for
 * the ray: entry and exit close (grazing), or two candidate entry times
 * close (the entry face, or for a gate whether the entry is inside the
 * opening, may change in FP32).  kdir (>= 1) scales the margins that come
 * from the ray direction's FP32 error (the pose's attitude conditioning).
 * Returns amb bits: 1|2 value, 2 gradient. */
static int prim_amb(const map_t *m, int id, const double *o, const double *d, double reach, double kdir)
{
    int flags = 0;
    if (fabs(prim_sdf(m, id, o)) < AMB_INSIDE) flags |= 3;
    if (id < m->ns) {
        const double *sp = m->sph + 4 * id;
        double oc[3] = {sp[0] - o[0], sp[1] - o[1], sp[2] - o[2]};
        double C = dot3(oc, oc) - sp[3] * sp[3];
        double b = dot3(d, oc);
        double disc = b * b - C;
        if (b > 0.0 && b - sqrt(fabs(disc)) < reach && fabs(disc) < kdir * AMB_DISC * (b * b > 1.0 ? b * b : 1.0))
            flags |= 3;
        return flags;
    }
    int k = id - m->ns;
    if (k < m->nb) {
        const double *bx = m->box + 6 * k;
        double tn = -OC_INF, tf = OC_INF;
        int ok = 1;
        for (int i = 0; i < 3; ++i) {
            if (d[i] == 0.0) { if (o[i] < bx[i] || o[i] > bx[3 + i]) ok = 0; continue; }
            double t1 = (bx[i] - o[i]) / d[i], t2 = (bx[3 + i] - o[i]) / d[i];
            double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
            if (lo > tn) tn = lo;
            if (hi < tf) tf = hi;
        }
        if (ok && tn > 0.0 && tn < reach && fabs(tf - tn) < kdir * AMB_SLAB) flags |= 3;
        return flags;
    }
    k -= m->nb;
    /* cylinders and gates: collect the interval end points and compare */
    double e[10];
    int ne = 0;
    if (k < m->nc) {
        const double *cy = m->cyl + 5 * k;
        double ex = o[0] - cy[0], ey = o[1] - cy[1];
        double a = d[0] * d[0] + d[1] * d[1], b = d[0] * ex + d[1] * ey;
        double cc = ex * ex + ey * ey - cy[2] * cy[2];
        if (a > 0.0) {
            double disc = b * b - a * cc;
            double sq = sqrt(fabs(disc));
            /* grazing the side: the two roots (nearly) coincide */
            if ((-b - sq) / a < reach && -b + sq > 0.0 && fabs(disc) < kdir * AMB_DISC * (b * b > a ? b * b : a))
                flags |= 3;
            if (disc >= 0.0) { e[ne++] = (-b - sq) / a; e[ne++] = (-b + sq) / a; }
        }
        if (d[2] != 0.0) { e[ne++] = (cy[3] - o[2]) / d[2]; e[ne++] = (cy[4] - o[2]) / d[2]; }
    } else {
        const double *g = m->gate + 7 * (k - m->nc);
        double uo[3], ud[3];
        gate_local(g, o, 0, uo);
        gate_local(g, d, 1, ud);
        double W = g[4] + g[5], half[3] = {g[6], W, W};
        for (int i = 0; i < 3; ++i)
            if (ud[i] != 0.0) {
                e[ne++] = (-half[i] - uo[i]) / ud[i];
                e[ne++] = (half[i] - uo[i]) / ud[i];
            }
        for (int i = 1; i < 3; ++i)
            if (ud[i] != 0.0) {
                e[ne++] = (-g[4] - uo[i]) / ud[i];
                e[ne++] = (g[4] - uo[i]) / ud[i];
            }
    }
    for (int i = 0; i < ne; ++i)
        for (int j = i + 1; j < ne; ++j) {
            double lo = e[i] < e[j] ? e[i] : e[j];
            if (lo > 0.0 && lo < reach && fabs(e[i] - e[j]) < kdir * AMB_EDGE * (lo > 1.0 ? lo : 1.0)) flags |= 3;
        }
    return flags;
}

/* One ray cast against every primitive of a map, brute force.  Returns t*
 * (+inf on a miss) and the hit id (lowest id among exact ties; -1 on a miss).
 * amb receives the flags of this ray, given the clamp distance tclamp in ray
 * length: bit 0 a value decision near its threshold (grazing, origin near a
 * surface), bit 1 a gradient decision near its threshold (second hit, range
 * clamp, box edge), bit 2 a value ill-conditioned in FP32, bit 3 a gradient
 * ill-conditioned under FP32 trajectory drift (near-grazing incidence), bit
 * 4 a gradient ill-conditioned under FP32 rounding of the pose alone (no
 * drift).  kdir (>= 1) is the attitude's conditioning at this pose: how much
 * the FP32 error of the body axes exceeds that of a well-conditioned
 * rotation (pose_kappa); it scales every margin that the ray direction's
 * error sets. */
static double cast_ray(const double *o, const double *d, const map_t *m, int *hit, double tclamp, int *amb,
                       double kdir)
{
    double best = OC_INF, second = OC_INF;
    int id = -1, flags = 0, aux = -1;
    const int np = map_count(m);
    for (int k = 0; k < np; ++k) {
        int ak;
        double t = prim_ray(m, k, o, d, &ak);
        if (t < best) { second = best; best = t; id = k; aux = ak; }
        else if (t < second) second = t;
    }
    /* near-degenerate decisions that could change the value in FP32 */
    double reach = (best < tclamp ? best : tclamp) + 1e-2;
    for (int k = 0; k < np; ++k) flags |= prim_amb(m, k, o, d, reach, kdir);
    /* gradient-only ambiguities: second hit close, range clamp, grazing,
     * entry through a box edge */
    if (best < OC_INF) {
        if (second - best < kdir * AMB_GAP) flags |= 2;
        if (fabs(best - tclamp) < AMB_RANGE) flags |= 2;
        double n[3];
        if (best > 0.0 && best < tclamp && prim_normal(m, id, o, d, best, aux, n)) {
            if (id >= m->ns && id < m->ns + m->nb) {
                /* two slab entry times within AMB_EDGE: the ray enters at an edge */
                const double *bx = m->box + 6 * (id - m->ns);
                double tl[3];
                for (int i = 0; i < 3; ++i) {
                    if (d[i] == 0.0) { tl[i] = -OC_INF; continue; }
                    double t1 = (bx[i] - o[i]) / d[i], t2 = (bx[3 + i] - o[i]) / d[i];
                    tl[i] = t1 < t2 ? t1 : t2;
                }
                for (int i = 0; i < 3; ++i)
                    if (i != aux && fabs(tl[i] - best) < kdir * AMB_EDGE * (best > 1.0 ? best : 1.0)) flags |= 2;
            }
            double nd = fabs(dot3(n, d));
            if (nd < AMB_GRAZE) flags |= 8;
            /* gradient -n/(n.d) of a curved hit turns by ~ dp/(r |n.d|) when
             * the trajectory drifts by dp (FP32 rollout): flag above 3e-4 */
            double rc = 0.0;  /* radius of curvature of a curved hit, 0 if flat */
            if (id < m->ns) rc = m->sph[4 * id + 3];
            if (id >= m->ns + m->nb && id < m->ns + m->nb + m->nc && aux == 0) rc = m->cyl[5 * (id - m->ns - m->nb) + 2];
            if (rc > 0.0 && DRIFT_POS / (rc * nd) > 3e-4) flags |= 8;
            /* rounding the pose to FP32 (direction COND_DIR kdir per
             * component, origin COND_ORG) moves the hit by dp = (COND_DIR kdir
             * t + COND_ORG) / |n.d|: the value is ill-conditioned when dp
             * exceeds half the depth tolerance; the gradient when its relative
             * change, dp / (r |n.d|) on a curved surface and COND_DIR kdir /
             * |n.d| on any, exceeds the gradient tolerance (1e-3) */
            double dp = (COND_DIR * kdir * best + COND_ORG) / nd;
            if (dp > COND_MAX) flags |= 4 | 8;
            if ((rc > 0.0 && dp / (rc * nd) > 1e-3) || COND_DIR * kdir / nd > 1e-3) flags |= 16;
        }
    }
    *hit = id;
    *amb = flags;
    return best;
}

/* -------------------------------------------------- obstacles and collisions */

/* Minimum signed distance from p to the map's primitives and the arg-min id
 * (lowest id among exact ties; -1 and +inf for an empty map).  gap receives
 * the distance between the two smallest values. */
static double sdf_min(const double *p, const map_t *m, int *id, double *gap)
{
    double best = OC_INF, second = OC_INF;
    int bi = -1;
    const int np = map_count(m);
    for (int k = 0; k < np; ++k) {
        double s = prim_sdf(m, k, p);
        if (s < best) { second = best; best = s; bi = k; }
        else if (s < second) second = s;
    }
    *id = bi;
    *gap = second - best;
    return best;
}

static void sdf_grad(const double *p, const map_t *m, int id, double *gp)
{
    if (id < m->ns) {
        const double *sp = m->sph + 4 * id;
        double d[3] = {p[0] - sp[0], p[1] - sp[1], p[2] - sp[2]};
        double n = norm3(d);
        for (int i = 0; i < 3; ++i) gp[i] = n > 0.0 ? d[i] / n : 0.0;
        return;
    }
    id -= m->ns;
    if (id < m->nb) { sdf_box_grad(p, m->box + 6 * id, gp); return; }
    id -= m->nb;
    if (id < m->nc) { sdf_cylinder_grad(p, m->cyl + 5 * id, gp); return; }
    sdf_gate_grad(p, m->gate + 7 * (id - m->nc), gp);
}

/* ------------------------------------------------------------ rollout state */

typedef struct {
    const oc_config *c;
    const oc_scene *sc;
    int D, A, NM, Rc, Rl;
    double *cam_dir, *cam_fac, *lid_dir;
} ctx_t;

static void ctx_init(ctx_t *x, const oc_config *c, const oc_scene *sc)
{
    x->c = c; x->sc = sc;
    x->D = oc_state_dim(c->model);
    x->A = oc_action_dim(c->model);
    x->NM = c->n_env * c->n_agent;
    x->Rc = c->cam_w > 0 ? c->cam_w * c->cam_h : 0;
    x->Rl = c->lid_ch > 0 ? c->lid_ch * c->lid_az : 0;
    x->cam_dir = x->Rc ? malloc(sizeof(double) * 3 * x->Rc) : NULL;
    x->cam_fac = x->Rc ? malloc(sizeof(double) * x->Rc) : NULL;
    x->lid_dir = x->Rl ? malloc(sizeof(double) * 3 * x->Rl) : NULL;
    if (x->Rc) oc_cam_dirs(c, x->cam_dir, x->cam_fac);
    if (x->Rl) oc_lidar_dirs(c, x->lid_dir);
}

static void ctx_free(ctx_t *x)
{
    free(x->cam_dir); free(x->cam_fac); free(x->lid_dir);
}

static void map_of(const ctx_t *x, int env, map_t *mp)
{
    const oc_scene *sc = x->sc;
    int m = sc->env_map[env];
    mp->sph = sc->spheres + 4 * sc->sph_off[m];
    mp->ns = sc->sph_off[m + 1] - sc->sph_off[m];
    mp->box = sc->boxes + 6 * sc->box_off[m];
    mp->nb = sc->box_off[m + 1] - sc->box_off[m];
    mp->cyl = sc->cylinders ? sc->cylinders + 5 * sc->cyl_off[m] : NULL;
    mp->nc = sc->cylinders ? sc->cyl_off[m + 1] - sc->cyl_off[m] : 0;
    mp->gate = sc->gates ? sc->gates + 7 * sc->gate_off[m] : NULL;
    mp->ng = sc->gates ? sc->gate_off[m + 1] - sc->gate_off[m] : 0;
}

static void dyn_step(const ctx_t *x, int env, const double *s, const double *a, double *o)
{
    if (x->c->model == OC_RIGID) { oc_rb_step(x->c, s, a, o); return; }
    if (x->c->model == OC_PMD) { oc_pmd_step(x->c, s, a, o); return; }
    if (x->c->model == OC_SIMPLE) { oc_simple_step(x->c, s, a, o); return; }
    double drag = x->sc->drag_env ? x->sc->drag_env[env] : x->c->drag;
    double lam = x->sc->lam_env ? x->sc->lam_env[env] : x->c->lam;
    oc_pm_step(x->c, drag, lam, s, a, o);
}

/* Render one agent: world ray = R * body ray, origin = position.  Camera
 * output is z-depth min(t* fac, range); lidar output is min(t*, range). */
static void render_agent(const ctx_t *x, int env, const double *s, double *depth, double *lidar,
                         int32_t *hc, int32_t *hl, uint8_t *ac, uint8_t *al)
{
    map_t mp;
    map_of(x, env, &mp);
    double o[3], R[9];
    int pf = oc_pose(x->c, s, o, R);
    double kdir = pose_kappa(x->c, s);
    for (int r = 0; r < x->Rc; ++r) {
        const double *db = x->cam_dir + 3 * r;
        double d[3];
        for (int i = 0; i < 3; ++i) d[i] = R[3 * i] * db[0] + R[3 * i + 1] * db[1] + R[3 * i + 2] * db[2];
        int id, amb;
        double tcl = x->c->cam_range / x->cam_fac[r];
        double t = cast_ray(o, d, &mp, &id, tcl, &amb, kdir);
        double z = t * x->cam_fac[r];
        if (depth) depth[r] = z < x->c->cam_range ? z : x->c->cam_range;
        hc[r] = id;
        ac[r] = (uint8_t)(amb | ((pf & 4) ? 3 : 0));
    }
    for (int r = 0; r < x->Rl; ++r) {
        const double *db = x->lid_dir + 3 * r;
        double d[3];
        for (int i = 0; i < 3; ++i) d[i] = R[3 * i] * db[0] + R[3 * i + 1] * db[1] + R[3 * i + 2] * db[2];
        int id, amb;
        double t = cast_ray(o, d, &mp, &id, x->c->lid_range, &amb, kdir);
        if (lidar) lidar[r] = t < x->c->lid_range ? t : x->c->lid_range;
        hl[r] = id;
        al[r] = (uint8_t)(amb | ((pf & 4) ? 3 : 0));
    }
}

/* Render the sensors of given states [NM][D] (no dynamics): used for the
 * observation of the initial state. */
int oc_render(const oc_config *c, const oc_scene *sc, const double *s, double *depth,
              double *lidar, int32_t *hit_cam, int32_t *hit_lid, uint8_t *amb_cam,
              uint8_t *amb_lid)
{
    ctx_t x;
    ctx_init(&x, c, sc);
    int M = c->n_agent;
    for (int i = 0; i < x.NM; ++i)
        render_agent(&x, i / M, s + (size_t)i * x.D,
                     depth ? depth + (size_t)i * x.Rc : NULL, lidar ? lidar + (size_t)i * x.Rl : NULL,
                     hit_cam + (size_t)i * x.Rc, hit_lid + (size_t)i * x.Rl,
                     amb_cam + (size_t)i * x.Rc, amb_lid + (size_t)i * x.Rl);
    ctx_free(&x);
    return 0;
}

/* ---------------------------------------------------- culling work count */

/* Bounding sphere (centre cb, radius) of primitive id of a map. */
static double prim_bound(const map_t *m, int id, double *cb)
{
    if (id < m->ns) {
        for (int i = 0; i < 3; ++i) cb[i] = m->sph[4 * id + i];
        return m->sph[4 * id + 3];
    }
    id -= m->ns;
    if (id < m->nb) {
        const double *b = m->box + 6 * id;
        double h2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            cb[i] = 0.5 * (b[i] + b[3 + i]);
            double h = 0.5 * (b[3 + i] - b[i]);
            h2 += h * h;
        }
        return sqrt(h2);
    }
    id -= m->nb;
    if (id < m->nc) {
        const double *cy = m->cyl + 5 * id;
        double hz = 0.5 * (cy[4] - cy[3]);
        cb[0] = cy[0]; cb[1] = cy[1]; cb[2] = 0.5 * (cy[3] + cy[4]);
        return sqrt(hz * hz + cy[2] * cy[2]);
    }
    const double *g = m->gate + 7 * (id - m->nc);
    double W = g[4] + g[5];
    for (int i = 0; i < 3; ++i) cb[i] = g[i];
    return sqrt(g[6] * g[6] + 2.0 * W * W);
}

/* Post-cull work of one render of the states s [NM][D] (Sec. III-B: each
 * sensor's rays are cast only against the primitives that its field of view
 * can reach).  The culling rule counted here is the one the CUDA path applies
 * with frustum culling (cull mode 1), restated in double precision from its
 * definition: a primitive is kept for an agent's sensor when its bounding
 * sphere (centre c, radius rho, relative position oc = c - o) either holds
 * the origin (|oc| <= rho + 1e-3) or lies within reach (|oc| - rho <= L +
 * 1e-3, L the longest unclamped ray: range / cos of the corner ray for the
 * camera, the range for the LiDAR) and meets the sensor's field of view with
 * a 1e-3 m margin: for the camera the four side planes of the pinhole
 * frustum (body frame, signed distance of the centre >= -(rho + 1e-3)); for
 * the LiDAR the elevation band widened by 1e-3 rad and by the sphere's
 * angular radius.  An agent whose origin lies in a primitive casts no test.
 * out[0] ray-sphere tests, out[1] tests of the other kinds, out[2] rays,
 * out[3] a bound on the tests that decisions within 1e-6 of a threshold (in
 * double precision) could move. */
int oc_cull_counts(const oc_config *c, const oc_scene *sc, const double *s, double *out)
{
    ctx_t x;
    ctx_init(&x, c, sc);
    const int M = c->n_agent;
    const double mg = 1e-3, eps = 1e-6;
    double th = tan(0.5 * c->cam_hfov), tv = th * (double)c->cam_h / (double)(c->cam_w > 0 ? c->cam_w : 1);
    double uc = (1.0 - 1.0 / (c->cam_w > 0 ? c->cam_w : 1)) * th, vc = (1.0 - 1.0 / (c->cam_h > 0 ? c->cam_h : 1)) * tv;
    double cam_len = c->cam_range * sqrt(1.0 + uc * uc + vc * vc);
    double c2 = 1.0 / sqrt(1.0 + th * th), c3 = 1.0 / sqrt(1.0 + tv * tv);
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    for (int i = 0; i < x.NM; ++i) {
        map_t mp;
        map_of(&x, i / M, &mp);
        double o[3], R[9];
        oc_pose(c, s + (size_t)i * x.D, o, R);
        const int np = map_count(&mp);
        /* origin inside a primitive (closed sets), and how close to a surface */
        int inside = 0;
        double near_surf = OC_INF;
        for (int k = 0; k < np; ++k) {
            double d = prim_sdf(&mp, k, o);
            if (d <= 0.0) inside = 1;
            if (fabs(d) < near_surf) near_surf = fabs(d);
        }
        for (int sen = 0; sen < 2; ++sen) {
            const int R_s = sen == 0 ? x.Rc : x.Rl;
            if (R_s == 0) continue;
            out[2] += R_s;
            const double len = sen == 0 ? cam_len : c->lid_range;
            long ks = 0, ko = 0, amb = 0;
            for (int k = 0; k < np; ++k) {
                double cb[3], oc[3], bx[3];
                double rho = prim_bound(&mp, k, cb);
                for (int j = 0; j < 3; ++j) oc[j] = cb[j] - o[j];
                for (int j = 0; j < 3; ++j) bx[j] = R[j] * oc[0] + R[3 + j] * oc[1] + R[6 + j] * oc[2];
                double L2 = dot3(oc, oc), r = rho + mg, rout = len + mg + rho;
                int near = L2 <= r * r, far = L2 > rout * rout, keep;
                int a = fabs(L2 - r * r) < eps * (L2 > 1.0 ? L2 : 1.0) || fabs(L2 - rout * rout) < eps * (L2 > 1.0 ? L2 : 1.0);
                if (sen == 0) {
                    double f[4] = {th * c2 * bx[0] - c2 * bx[1], th * c2 * bx[0] + c2 * bx[1],
                                   tv * c3 * bx[0] - c3 * bx[2], tv * c3 * bx[0] + c3 * bx[2]};
                    int in = 1;
                    for (int q = 0; q < 4; ++q) {
                        if (f[q] < -r) in = 0;
                        if (fabs(f[q] + r) < eps * (1.0 + sqrt(L2))) a = 1;
                    }
                    keep = near || (!far && in);
                } else {
                    double L = sqrt(L2);
                    if (near) keep = 1;
                    else if (far) keep = 0;
                    else {
                        double el = asin(clamp1(bx[2] / L)), del = asin(r / L < 1.0 ? r / L : 1.0);
                        double lo = c->lid_elev_lo - mg, hi = c->lid_elev_hi + mg;
                        keep = el - del <= hi && el + del >= lo;
                        if (fabs(el - del - hi) < eps || fabs(el + del - lo) < eps) a = 1;
                    }
                }
                if (keep) {
                    if (k < mp.ns) ++ks;
                    else ++ko;
                }
                amb += a;
            }
            if (inside) {
                ks = ko = 0;
            }
            out[0] += (double)R_s * ks;
            out[1] += (double)R_s * ko;
            out[3] += (double)R_s * (near_surf < eps ? np : amb);
        }
    }
    ctx_free(&x);
    return 0;
}

/* ------------------------------------------------------------------ IMU */

/* IMU readout of one agent after a step (Sec. III-B), noise-free: the
 * specific force f = R^T (v' - g) of the model's translational dynamics and
 * the body angular rate, both in the body frame of the new state s1 (before
 * any reset), with the step's action a held over the step.
 *   rigid (Eq. 1):      f = (T/m) e3 - D R^T v,   omega = the state's omega
 *   point mass (Eq. 3): f = R^T (a - d v)          (a: the lagged thrust)
 *   discrete (Eq. 4):   f = R^T u                  (u: the command in force)
 *   simplified (Eq. 2): f = c e3,                  omega = the commanded rates
 * The point-mass attitude has no rate state, so its angular rate is that of
 * the attitude change over the step, vee(A - A^T) / (2 dt), A = R0^T R1, with
 * R0 the attitude of s0, the state the step started from. */
static void imu_eval(const oc_config *c, double drag, const double *s0, const double *a,
                     const double *s1, double *out)
{
    double o[3], R1[9];
    oc_pose(c, s1, o, R1);
    if (c->model == OC_RIGID) {
        const double *v = s1 + 7, *w = s1 + 10;
        double T = c->mass * c->gravity * (1.0 + clamp1(a[0]));
        for (int j = 0; j < 3; ++j) {
            double vb = R1[j] * v[0] + R1[3 + j] * v[1] + R1[6 + j] * v[2];
            out[j] = (j == 2 ? T / c->mass : 0.0) - c->drag_body[j] * vb;
            out[3 + j] = w[j];
        }
        return;
    }
    if (c->model == OC_SIMPLE) {
        for (int j = 0; j < 3; ++j) {
            out[j] = j == 2 ? c->gravity * (1.0 + clamp1(a[0])) : 0.0;
            out[3 + j] = c->rate_scale[j] * clamp1(a[1 + j]);
        }
        return;
    }
    double acc[3], R0[9], A[9];
    for (int i = 0; i < 3; ++i)
        acc[i] = c->model == OC_PMD ? s1[6 + i] : s1[6 + i] - drag * s1[3 + i];
    for (int j = 0; j < 3; ++j) out[j] = R1[j] * acc[0] + R1[3 + j] * acc[1] + R1[6 + j] * acc[2];
    oc_pose(c, s0, o, R0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = R0[i] * R1[j] + R0[3 + i] * R1[3 + j] + R0[6 + i] * R1[6 + j];
    out[3] = (A[7] - A[5]) / (2.0 * c->dt);
    out[4] = (A[2] - A[6]) / (2.0 * c->dt);
    out[5] = (A[3] - A[1]) / (2.0 * c->dt);
}

/* IMU after a reset: the new state read as held at rest (f = -R^T g, the
 * rigid body's rate state, else no rate); carries no cotangent. */
static void imu_reset(const oc_config *c, const double *s, double *out)
{
    double o[3], R[9];
    oc_pose(c, s, o, R);
    for (int j = 0; j < 3; ++j) {
        out[j] = R[6 + j] * c->gravity;
        out[3 + j] = c->model == OC_RIGID ? s[10 + j] : 0.0;
    }
}

/* ---------------------------------------------------------------- racing */

/* Local normal coordinate u_n of point x and, at the crossing of the gate's
 * centre plane on the segment x0 -> x1, whether it lies inside the opening.
 * A gate is passed when u_n goes from negative to non-negative along the
 * step (travel along the normal) and the crossing point is in the opening. */
static int gate_passed(const double *g, const double *x0, const double *x1, int *amb)
{
    double u0[3], u1[3];
    gate_local(g, x0, 0, u0);
    gate_local(g, x1, 0, u1);
    if (fabs(u0[0]) < AMB_STEP || fabs(u1[0]) < AMB_STEP) *amb |= 1;
    if (!(u0[0] < 0.0 && u1[0] >= 0.0)) return 0;
    double f = -u0[0] / (u1[0] - u0[0]);
    double ul = u0[1] + f * (u1[1] - u0[1]), uz = u0[2] + f * (u1[2] - u0[2]);
    if (fabs(fabs(ul) - g[4]) < AMB_STEP || fabs(fabs(uz) - g[4]) < AMB_STEP) *amb |= 1;
    return fabs(ul) < g[4] && fabs(uz) < g[4];
}

/* One environment step for all agents of env (Sec. III-C, III-D):
 * dynamics -> collision and rewards on the new state -> termination ->
 * reset of the whole environment from the pool -> sensor rendering of the
 * (possibly reset) new state.  Collision: obstacle SDF < r_quad, position
 * outside [bound_lo, bound_hi], or another agent of the env closer than
 * d_agent.  R_ctrl = -w_pos |e|^(1 or 2) - w_obs relu(d_safe - sdf)^2
 *                    - w_act |action|^2 - w_agent sum_j relu(d_agent - d_ij)^2,
 * R_goal = -1 on collision, +1 within success_radius of the target, else 0.
 * Racing (task 1): each agent targets gate k of the map's ordered gates;
 * the position term becomes the progress w_pos (|p_t - g_k| - |p_{t+1} - g_k|)
 * towards that gate's centre, R_goal = +1 when the step passes the gate
 * (then k advances, cyclically), -1 on collision; a reset restarts at gate 0.
 * The IMU (when ex->imu is set) reads the new state after a possible reset. */
static void env_step(const ctx_t *x, int env, int t, const double *s_t, const double *act_t,
                     int32_t *pool_k, double *s_next, double *spre, double *r_ctrl,
                     int8_t *r_goal, uint8_t *done, double *depth, double *lidar,
                     int32_t *hc, int32_t *hl, uint8_t *ac, uint8_t *al, uint8_t *amb_step,
                     int32_t *sdf_id, const oc_extra *ex)
{
    const oc_config *c = x->c;
    int M = c->n_agent, D = x->D, A = x->A;
    map_t mp;
    map_of(x, env, &mp);
    int i0 = env * M;
    int any = 0;
    int *coll = calloc((size_t)M, sizeof(int));
    for (int m = 0; m < M; ++m) {
        int i = i0 + m;
        dyn_step(x, env, s_t + (size_t)i * D, act_t + (size_t)i * A, spre + (size_t)i * D);
    }
    for (int m = 0; m < M; ++m) {
        int i = i0 + m, id, flags = 0;
        const double *p = spre + (size_t)i * D;
        const double *a = act_t + (size_t)i * A;
        double gap;
        double sd = sdf_min(p, &mp, &id, &gap);
        sdf_id[i] = id;
        int col = sd < c->r_quad;
        if (fabs(sd - c->r_quad) < AMB_STEP) flags |= 1;
        for (int k = 0; k < 3; ++k) {
            if (p[k] < c->bound_lo[k] || p[k] > c->bound_hi[k]) col = 1;
            if (fabs(p[k] - c->bound_lo[k]) < AMB_STEP || fabs(p[k] - c->bound_hi[k]) < AMB_STEP) flags |= 1;
        }
        double pair = 0.0;
        for (int n = 0; n < M; ++n) {
            if (n == m) continue;
            const double *q = spre + (size_t)(i0 + n) * D;
            double dd[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
            double dij = norm3(dd);
            if (dij < c->d_agent) col = 1;
            if (fabs(dij - c->d_agent) < AMB_STEP) flags |= 1;
            pair += relu(c->d_agent - dij) * relu(c->d_agent - dij);
        }
        double ob = (c->w_obs != 0.0 && sd < OC_INF) ? relu(c->d_safe - sd) : 0.0;
        double aa = 0.0;
        for (int k = 0; k < A; ++k) aa += a[k] * a[k];
        double ne = 1.0;
        if (c->task == 1) {
            const int gk = ex->gate_k[i];
            const double *g = mp.gate + 7 * gk;
            const double *p0 = s_t + (size_t)i * D;
            double e0[3] = {p0[0] - g[0], p0[1] - g[1], p0[2] - g[2]};
            double e1[3] = {p[0] - g[0], p[1] - g[1], p[2] - g[2]};
            ne = norm3(e1);
            if (ex->gate_tape) ex->gate_tape[(size_t)t * x->NM + i] = gk;
            int passed = gate_passed(g, p0, p, &flags);
            r_ctrl[i] = c->w_pos * (norm3(e0) - ne) - c->w_obs * ob * ob - c->w_act * aa - c->w_agent * pair;
            r_goal[i] = (int8_t)(col ? -1 : (passed ? 1 : 0));
            if (passed) ex->gate_k[i] = (gk + 1) % mp.ng;
            if (norm3(e0) < 1e-6) flags |= 2;
        } else {
            const double *tg = x->sc->targets + 3 * (size_t)i;
            double e[3] = {p[0] - tg[0], p[1] - tg[1], p[2] - tg[2]};
            ne = norm3(e);
            double pos = c->pos_sq ? ne * ne : ne;
            r_ctrl[i] = -c->w_pos * pos - c->w_obs * ob * ob - c->w_act * aa - c->w_agent * pair;
            r_goal[i] = (int8_t)(col ? -1 : (ne < c->success_radius ? 1 : 0));
            if (fabs(ne - c->success_radius) < AMB_STEP) flags |= 1;
        }
        /* gradient kinks: arg-min tie of an active obstacle term, norm at 0,
         * action clip boundary, box SDF on its medial axis */
        if (ob > 0.0 && gap < AMB_STEP) flags |= 2;
        if ((!c->pos_sq || c->task == 1) && ne < 1e-6) flags |= 2;
        for (int k = 0; k < A; ++k)
            if (fabs(fabs(a[k]) - 1.0) < 1e-9) flags |= 2;
        amb_step[i] = (uint8_t)flags;
        coll[m] = col;
        any |= col;
    }
    int dn = c->terminate && any;
    for (int m = 0; m < M; ++m) {
        int i = i0 + m;
        done[i] = (uint8_t)dn;
        if (dn && c->pool_size > 0) {
            int k = pool_k[env] % c->pool_size;
            memcpy(s_next + (size_t)i * D, x->sc->pool + ((size_t)k * x->NM + i) * D, sizeof(double) * D);
        } else {
            memcpy(s_next + (size_t)i * D, spre + (size_t)i * D, sizeof(double) * D);
        }
    }
    if (dn) pool_k[env] += 1;
    if (dn && c->task == 1)
        for (int m = 0; m < M; ++m) ex->gate_k[i0 + m] = 0;
    if (ex && ex->imu) {
        double drag = x->sc->drag_env ? x->sc->drag_env[env] : c->drag;
        for (int m = 0; m < M; ++m) {
            int i = i0 + m;
            size_t o6 = ((size_t)t * x->NM + i) * 6;
            double *out = ex->imu + o6;
            if (dn) imu_reset(c, s_next + (size_t)i * D, out);
            else imu_eval(c, drag, s_t + (size_t)i * D, act_t + (size_t)i * A, spre + (size_t)i * D, out);
            if (ex->imu_noise) {
                const double *z = ex->imu_noise + 2 * o6;
                double *b = ex->imu_bias + (size_t)i * 6;
                if (dn) memset(b, 0, 6 * sizeof(double));
                for (int k = 0; k < 6; ++k) {
                    out[k] += b[k] + c->imu_noise[k / 3] * z[k];
                    b[k] += c->imu_walk[k / 3] * sqrt(c->dt) * z[6 + k];
                }
            }
        }
    }
    for (int m = 0; m < M; ++m) {
        int i = i0 + m;
        double o[3], R[9];
        if ((c->model == OC_PM || c->model == OC_PMD) && (oc_pose(c, s_next + (size_t)i * D, o, R) & 4))
            amb_step[i] |= 4;
        render_agent(x, env, s_next + (size_t)i * D,
                     depth ? depth + (size_t)i * x->Rc : NULL, lidar ? lidar + (size_t)i * x->Rl : NULL,
                     hc + (size_t)i * x->Rc, hl + (size_t)i * x->Rl,
                     ac + (size_t)i * x->Rc, al + (size_t)i * x->Rl);
    }
    (void)t;
    free(coll);
}

/* Rollout over the horizon.  states [T+1][NM][D] receives s_0..s_T (after
 * resets), spre [T][NM][D] the states before reset.  pool_k [N] is the reset
 * counter of each env, read and advanced.  depth/lidar and their hit ids and
 * flags are [T][NM][R]; output t is the observation of s_{t+1}.  ex holds the
 * racing and IMU state (NULL: neither; racing requires ex->gate_k).
 * n_threads parallelises over environments only. */
int oc_rollout(const oc_config *c, const oc_scene *sc, const double *s0, int32_t *pool_k,
               const double *act, double *states, double *spre, double *r_ctrl, int8_t *r_goal,
               uint8_t *done, double *depth, double *lidar, int32_t *hit_cam, int32_t *hit_lid,
               uint8_t *amb_cam, uint8_t *amb_lid, uint8_t *amb_step, int32_t *sdf_id,
               const oc_extra *ex, int n_threads)
{
    ctx_t x;
    ctx_init(&x, c, sc);
    int N = c->n_env, M = c->n_agent, T = c->horizon, D = x.D, A = x.A, NM = x.NM;
    memcpy(states, s0, sizeof(double) * (size_t)NM * D);
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int env = 0; env < N; ++env) {
        for (int t = 0; t < T; ++t) {
            size_t sT = (size_t)t * NM;
            env_step(&x, env, t, states + sT * D, act + sT * A, pool_k,
                     states + (sT + NM) * D, spre + sT * D, r_ctrl + sT, r_goal + sT, done + sT,
                     depth ? depth + sT * x.Rc : NULL, lidar ? lidar + sT * x.Rl : NULL,
                     hit_cam + sT * x.Rc, hit_lid + sT * x.Rl, amb_cam + sT * x.Rc,
                     amb_lid + sT * x.Rl, amb_step + sT, sdf_id + sT, ex);
        }
    }
    (void)M;
    ctx_free(&x);
    return 0;
}

/* ------------------------------------------------------------------ adjoint */

/* VJP of the point-mass step (Eq. 3, explicit Euler): given the cotangent go of
 * the new state, accumulate into gs (old state) and ga (raw action). */
static void pm_step_vjp(const oc_config *c, double drag, double lam, const double *s,
                        const double *act, const double *go, double *gs, double *ga)
{
    double al = c->ema_alpha, dt = c->dt;
    for (int i = 0; i < 3; ++i) {
        double gp = go[i], gv = go[3 + i], gA = go[6 + i], ge = go[9 + i];
        gv += al * ge;                 /* ema' = (1-al) ema + al v' */
        gs[9 + i] += (1.0 - al) * ge;
        gs[i] += gp;                   /* p' = p + dt v */
        gs[3 + i] += dt * gp;
        gs[3 + i] += (1.0 - dt * drag) * gv; /* v' = v + dt (a + g - d v) */
        gs[6 + i] += dt * gv;
        gs[6 + i] += (1.0 - dt * lam) * gA;  /* a' = a + dt lam (u - a) */
        double gu = dt * lam * gA;
        ga[i] += c->act_scale * dclamp1(act[i]) * gu;
    }
    (void)s;
}

/* VJP of the discrete point-mass step (Eq. 4). */
static void pmd_step_vjp(const oc_config *c, const double *act, const double *go, double *gs, double *ga)
{
    double al = c->ema_alpha, dt = c->dt;
    for (int i = 0; i < 3; ++i) {
        double gp = go[i], gv = go[3 + i], gu1 = go[6 + i], ge = go[9 + i];
        gv += al * ge;
        gs[9 + i] += (1.0 - al) * ge;
        gs[i] += gp;                                 /* p' = p + v dt + 1/2 (u + g) dt^2 */
        gs[3 + i] += dt * gp + gv;                   /* v' = v + 1/2 (u + u1 + 2 g) dt */
        gs[6 + i] += 0.5 * dt * dt * gp + 0.5 * dt * gv;
        gu1 += 0.5 * dt * gv;
        ga[i] += c->act_scale * dclamp1(act[i]) * gu1;
    }
}

/* VJP of Gram-Schmidt (columns of Rt -> Ro) given the cotangent gRo. */
static void gram_schmidt_vjp(const double *Rt, const double *gRo, double *gRt)
{
    double u0[3] = {Rt[0], Rt[3], Rt[6]}, u1[3] = {Rt[1], Rt[4], Rt[7]};
    double n0 = norm3(u0), x[3], wv[3], y[3];
    for (int i = 0; i < 3; ++i) x[i] = u0[i] / n0;
    double sx = dot3(x, u1);
    for (int i = 0; i < 3; ++i) wv[i] = u1[i] - sx * x[i];
    double n1 = norm3(wv);
    for (int i = 0; i < 3; ++i) y[i] = wv[i] / n1;
    double gx[3] = {gRo[0], gRo[3], gRo[6]}, gy[3] = {gRo[1], gRo[4], gRo[7]}, gz[3] = {gRo[2], gRo[5], gRo[8]};
    double t[3];
    cross3(y, gz, t);                   /* z = x cross y */
    for (int i = 0; i < 3; ++i) gx[i] += t[i];
    cross3(gz, x, t);
    for (int i = 0; i < 3; ++i) gy[i] += t[i];
    double yg = dot3(y, gy), gw[3];     /* y = w / |w| */
    for (int i = 0; i < 3; ++i) gw[i] = (gy[i] - y[i] * yg) / n1;
    double xg = dot3(x, gw), gu1[3];    /* w = u1 - (x.u1) x */
    for (int i = 0; i < 3; ++i) {
        gu1[i] = gw[i] - x[i] * xg;
        gx[i] -= xg * u1[i] + sx * gw[i];
    }
    double xx = dot3(x, gx), gu0[3];    /* x = u0 / |u0| */
    for (int i = 0; i < 3; ++i) gu0[i] = (gx[i] - x[i] * xx) / n0;
    for (int i = 0; i < 3; ++i) {
        gRt[3 * i] = gu0[i];
        gRt[3 * i + 1] = gu1[i];
        gRt[3 * i + 2] = 0.0;
    }
}

/* VJP of the simplified quadrotor step (Eq. 2, explicit Euler, Gram-Schmidt). */
static void simple_step_vjp(const oc_config *c, const double *s, const double *act, const double *go, double *gs,
                            double *ga)
{
    const double *R = s + 6;
    double Rt[9], w[3], cth, gRt[9];
    simple_pre(c, s, act, Rt, w, &cth);
    const double dt = c->dt;
    for (int i = 0; i < 3; ++i) {
        gs[i] += go[i];                      /* p' = p + dt v */
        gs[3 + i] += dt * go[i] + go[3 + i]; /* v' = v + dt (R e3 c + g) */
    }
    double gc = 0.0;
    for (int i = 0; i < 3; ++i) {
        gs[6 + 3 * i + 2] += dt * cth * go[3 + i];
        gc += dt * R[3 * i + 2] * go[3 + i];
    }
    gram_schmidt_vjp(Rt, go + 6, gRt);
    /* Rt = R (I + dt [w]_x): gR += gRt (I + dt [w]_x)^T = gRt (I - dt [w]_x) */
    const double W[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += gRt[3 * i + k] * W[3 * j + k];
            gs[6 + 3 * i + j] += gRt[3 * i + j] + dt * acc;
        }
    /* w: M = R^T gRt; dL/dw1 = dt (M21 - M12), dw2 = dt (M02 - M20), dw3 = dt (M10 - M01) */
    double Mt[9];
    for (int a2 = 0; a2 < 3; ++a2)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * k + a2] * gRt[3 * k + b];
            Mt[3 * a2 + b] = acc;
        }
    double gw[3] = {dt * (Mt[7] - Mt[5]), dt * (Mt[2] - Mt[6]), dt * (Mt[3] - Mt[1])};
    ga[0] += c->gravity * dclamp1(act[0]) * gc;
    for (int i = 0; i < 3; ++i) ga[1 + i] += c->rate_scale[i] * dclamp1(act[1 + i]) * gw[i];
}

/* VJP of the rigid-body step (Eq. 1 with the rate controller, explicit Euler,
 * quaternion renormalisation). */
static void rb_step_vjp(const oc_config *c, const double *s, const double *act, const double *go,
                        double *gs, double *ga)
{
    const double *q = s + 3, *v = s + 7, *w = s + 10;
    const double *J = c->inertia;
    double dt = c->dt, m = c->mass;
    /* recompute the forward intermediates */
    double T = m * c->gravity * (1.0 + clamp1(act[0]));
    double R[9], vb[3], dvb[3], Jw[3], qw[4] = {0.0, w[0], w[1], w[2]}, qd[4], qt[4];
    oc_quat_to_rot(q, R);
    for (int j = 0; j < 3; ++j) vb[j] = R[0 + j] * v[0] + R[3 + j] * v[1] + R[6 + j] * v[2];
    for (int j = 0; j < 3; ++j) dvb[j] = c->drag_body[j] * vb[j];
    for (int i = 0; i < 3; ++i) Jw[i] = J[i] * w[i];
    quat_mul(q, qw, qd);
    for (int k = 0; k < 4; ++k) qt[k] = q[k] + dt * 0.5 * qd[k];
    double nq = sqrt(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
    double qn[4] = {qt[0] / nq, qt[1] / nq, qt[2] / nq, qt[3] / nq};

    const double *gp = go, *gqn = go + 3, *gvn = go + 7, *gwn = go + 10;
    double *gsp = gs, *gsq = gs + 3, *gsv = gs + 7, *gsw = gs + 10;
    /* p' = p + dt v */
    for (int i = 0; i < 3; ++i) { gsp[i] += gp[i]; gsv[i] += dt * gp[i]; }
    /* v' = v + dt vd */
    double gvd[3];
    for (int i = 0; i < 3; ++i) { gsv[i] += gvn[i]; gvd[i] = dt * gvn[i]; }
    /* q' = qt / |qt|, qt = q + dt/2 qd */
    double qg = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
    double gqt[4], gqd[4];
    for (int k = 0; k < 4; ++k) gqt[k] = (gqn[k] - qn[k] * qg) / nq;
    for (int k = 0; k < 4; ++k) { gsq[k] += gqt[k]; gqd[k] = 0.5 * dt * gqt[k]; }
    /* omega' = omega + dt wd */
    double gwd[3];
    for (int i = 0; i < 3; ++i) { gsw[i] += gwn[i]; gwd[i] = dt * gwn[i]; }
    /* qd = q (x) (0, w): w-part -v.w, vector part q_w w + v x w */
    {
        double vq[3] = {q[1], q[2], q[3]}, gvec[3] = {gqd[1], gqd[2], gqd[3]}, t3[3];
        gsq[0] += dot3(gvec, w);
        cross3(w, gvec, t3);
        for (int i = 0; i < 3; ++i) gsq[1 + i] += -gqd[0] * w[i] + t3[i];
        cross3(gvec, vq, t3);
        for (int i = 0; i < 3; ++i) gsw[i] += -gqd[0] * vq[i] + q[0] * gvec[i] + t3[i];
    }
    /* vd = g + (T/m) R e3 - R dvb, dvb = Dd (R^T v) */
    double gR[9] = {0}, gT = 0.0, gdvb[3], gvb[3];
    for (int i = 0; i < 3; ++i) {
        gT += R[3 * i + 2] * gvd[i] / m;
        gR[3 * i + 2] += (T / m) * gvd[i];
        for (int j = 0; j < 3; ++j) gR[3 * i + j] += -gvd[i] * dvb[j];
    }
    for (int j = 0; j < 3; ++j) gdvb[j] = -(R[0 + j] * gvd[0] + R[3 + j] * gvd[1] + R[6 + j] * gvd[2]);
    for (int j = 0; j < 3; ++j) gvb[j] = c->drag_body[j] * gdvb[j];
    for (int i = 0; i < 3; ++i) {
        gsv[i] += R[3 * i] * gvb[0] + R[3 * i + 1] * gvb[1] + R[3 * i + 2] * gvb[2];
        for (int j = 0; j < 3; ++j) gR[3 * i + j] += v[i] * gvb[j];
    }
    quat_to_rot_vjp(q, gR, gsq);
    /* wd = (tau - gy) / J; tau = J K (wc - w) + gy; gy = w x Jw */
    double gtau[3], ggy[3], gwc[3], t3[3];
    for (int i = 0; i < 3; ++i) { gtau[i] = gwd[i] / J[i]; ggy[i] = -gwd[i] / J[i]; }
    for (int i = 0; i < 3; ++i) {
        gwc[i] = J[i] * c->k_rate[i] * gtau[i];
        gsw[i] += -J[i] * c->k_rate[i] * gtau[i];
        ggy[i] += gtau[i];
    }
    cross3(Jw, ggy, t3);
    for (int i = 0; i < 3; ++i) gsw[i] += t3[i];
    cross3(ggy, w, t3);
    for (int i = 0; i < 3; ++i) gsw[i] += J[i] * t3[i];
    /* T = m g (1 + clip a0), wc = rate_scale clip(a1..3) */
    ga[0] += m * c->gravity * dclamp1(act[0]) * gT;
    for (int i = 0; i < 3; ++i) ga[1 + i] += c->rate_scale[i] * dclamp1(act[1 + i]) * gwc[i];
}

/* VJP of the sensor pose: gR (row-major) and go (origin) into gs. */
static void pose_vjp(const oc_config *c, const double *s, const double *go, const double *gR,
                     double *gs)
{
    for (int i = 0; i < 3; ++i) gs[i] += go[i];
    if (c->model == OC_RIGID) { quat_to_rot_vjp(s + 3, gR, gs + 3); return; }
    if (c->model == OC_SIMPLE) {
        for (int k = 0; k < 9; ++k) gs[6 + k] += gR[k];
        return;
    }
    const double *a = s + 6, *e = s + 9;
    double z[3], hp[3], x[3], h[3];
    double na = norm3(a);
    int zfb = na < 1e-6;
    if (zfb) { z[0] = 0; z[1] = 0; z[2] = 1; }
    else for (int i = 0; i < 3; ++i) z[i] = a[i] / na;
    h[0] = e[0]; h[1] = e[1]; h[2] = 0.0;
    double hz = dot3(h, z);
    for (int i = 0; i < 3; ++i) hp[i] = h[i] - hz * z[i];
    double nh = norm3(hp);
    int hfb = 0;
    if (nh < 1e-6) {
        hfb = 1;
        h[0] = 1; h[1] = 0; h[2] = 0;
        hz = dot3(h, z);
        for (int i = 0; i < 3; ++i) hp[i] = h[i] - hz * z[i];
        nh = norm3(hp);
        if (nh < 1e-6) {
            h[0] = 0; h[1] = 1; h[2] = 0;
            hz = dot3(h, z);
            for (int i = 0; i < 3; ++i) hp[i] = h[i] - hz * z[i];
            nh = norm3(hp);
        }
    }
    for (int i = 0; i < 3; ++i) x[i] = hp[i] / nh;
    double gx[3], gy[3], gz[3], t3[3];
    for (int i = 0; i < 3; ++i) { gx[i] = gR[3 * i]; gy[i] = gR[3 * i + 1]; gz[i] = gR[3 * i + 2]; }
    /* y = z x x */
    cross3(x, gy, t3);
    for (int i = 0; i < 3; ++i) gz[i] += t3[i];
    cross3(gy, z, t3);
    for (int i = 0; i < 3; ++i) gx[i] += t3[i];
    /* x = hp / |hp| */
    double xg = dot3(x, gx), ghp[3];
    for (int i = 0; i < 3; ++i) ghp[i] = (gx[i] - x[i] * xg) / nh;
    /* hp = h - (h.z) z */
    double zg = dot3(z, ghp);
    for (int i = 0; i < 3; ++i) gz[i] += -hz * ghp[i] - h[i] * zg;
    if (!hfb) {
        gs[9] += ghp[0] - z[0] * zg;
        gs[10] += ghp[1] - z[1] * zg;
    }
    /* z = a / |a| */
    if (!zfb) {
        double zz = dot3(z, gz);
        for (int i = 0; i < 3; ++i) gs[6 + i] += (gz[i] - z[i] * zz) / na;
    }
}

/* VJP of imu_eval: the cotangent g [6] of the readout into gs0 (the state
 * the step started from), gs1 (the new state before reset) and ga (the raw
 * action). */
static void imu_vjp(const oc_config *c, double drag, const double *s0, const double *a, const double *s1,
                    const double *g, double *gs0, double *gs1, double *ga)
{
    double o[3], R1[9], gR1[9] = {0}, zero[3] = {0.0, 0.0, 0.0};
    oc_pose(c, s1, o, R1);
    if (c->model == OC_RIGID) {
        /* f_j = g (1 + clip(a0)) [j = z] - D_j sum_i R_ij v_i */
        const double *v = s1 + 7;
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                gR1[3 * i + j] += -c->drag_body[j] * v[i] * g[j];
                gs1[7 + i] += -c->drag_body[j] * R1[3 * i + j] * g[j];
            }
        ga[0] += c->gravity * dclamp1(a[0]) * g[2];
        for (int j = 0; j < 3; ++j) gs1[10 + j] += g[3 + j];
        pose_vjp(c, s1, zero, gR1, gs1);
        return;
    }
    if (c->model == OC_SIMPLE) {
        ga[0] += c->gravity * dclamp1(a[0]) * g[2];
        for (int j = 0; j < 3; ++j) ga[1 + j] += c->rate_scale[j] * dclamp1(a[1 + j]) * g[3 + j];
        return;
    }
    /* f_j = sum_i R1_ij acc_i, acc = a_state - d v (continuous) or u (discrete) */
    double acc[3], gacc[3] = {0.0, 0.0, 0.0}, R0[9], gR0[9] = {0}, gA[9] = {0};
    for (int i = 0; i < 3; ++i) acc[i] = c->model == OC_PMD ? s1[6 + i] : s1[6 + i] - drag * s1[3 + i];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            gR1[3 * i + j] += acc[i] * g[j];
            gacc[i] += R1[3 * i + j] * g[j];
        }
    for (int i = 0; i < 3; ++i) {
        gs1[6 + i] += gacc[i];
        if (c->model != OC_PMD) gs1[3 + i] += -drag * gacc[i];
    }
    /* omega = vee(A - A^T) / (2 dt), A_ij = sum_k R0_ki R1_kj */
    oc_pose(c, s0, o, R0);
    double h = 1.0 / (2.0 * c->dt);
    gA[7] += h * g[3]; gA[5] -= h * g[3];
    gA[2] += h * g[4]; gA[6] -= h * g[4];
    gA[3] += h * g[5]; gA[1] -= h * g[5];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                gR0[3 * k + i] += gA[3 * i + j] * R1[3 * k + j];
                gR1[3 * k + j] += gA[3 * i + j] * R0[3 * k + i];
            }
    pose_vjp(c, s1, zero, gR1, gs1);
    pose_vjp(c, s0, zero, gR0, gs0);
}

/* VJP of one ray's output w.r.t. origin o and world direction d.  g is the
 * cotangent of the output, fac the factor from t* to the output (z-depth
 * factor or 1), clampv the output clamp.  Zero on a miss, a clamped output,
 * or an origin inside a primitive (t* = 0).  The hit-point normal n gives
 * dt/do = -n / (n.d) and dt/dd = -t n / (n.d). */
static void ray_vjp(const double *o, const double *d, const map_t *m, int id, double g, double fac,
                    double clampv, double *go, double *gd)
{
    if (id < 0 || g == 0.0) return;
    int aux;
    double n[3];
    double t = prim_ray(m, id, o, d, &aux);
    if (!(t > 0.0) || t * fac >= clampv) return;
    if (!prim_normal(m, id, o, d, t, aux, n)) return;
    double nd = dot3(n, d);
    double gt = g * fac;
    for (int i = 0; i < 3; ++i) {
        go[i] += gt * (-n[i] / nd);
        gd[i] += gt * (-t * n[i] / nd);
    }
}

/* render VJP of one agent: accumulates into gs (state cotangent). */
static void render_vjp(const ctx_t *x, int env, const double *s, const int32_t *hc,
                       const int32_t *hl, const double *gdep, const double *glid, double *gs)
{
    map_t mp;
    map_of(x, env, &mp);
    double o[3], R[9], go[3] = {0, 0, 0}, gR[9] = {0};
    oc_pose(x->c, s, o, R);
    for (int r = 0; gdep && r < x->Rc; ++r) {
        const double *db = x->cam_dir + 3 * r;
        double d[3], gd[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) d[i] = R[3 * i] * db[0] + R[3 * i + 1] * db[1] + R[3 * i + 2] * db[2];
        ray_vjp(o, d, &mp, hc[r], gdep[r], x->cam_fac[r], x->c->cam_range, go, gd);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) gR[3 * i + j] += gd[i] * db[j];
    }
    for (int r = 0; glid && r < x->Rl; ++r) {
        const double *db = x->lid_dir + 3 * r;
        double d[3], gd[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) d[i] = R[3 * i] * db[0] + R[3 * i + 1] * db[1] + R[3 * i + 2] * db[2];
        ray_vjp(o, d, &mp, hl[r], glid[r], 1.0, x->c->lid_range, go, gd);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) gR[3 * i + j] += gd[i] * db[j];
    }
    pose_vjp(x->c, s, go, gR, gs);
}

/* Adjoint of the rollout (Eq. 5 applied step by step, reverse order).  Inputs
 * are the actions and the records of oc_rollout; cotangents g_r [T][NM] of
 * R_ctrl, g_depth / g_lidar [T][NM][R] (NULL = zero), g_sT [NM][D] of the
 * final state (NULL = zero), g_imu [T][NM][6] of the IMU readout (NULL =
 * zero); gate_tape [T][NM] the racing record (task 1).  Outputs g_a
 * [T][NM][A] and g_s0 [NM][D].
 * A reset replaces the state, so no cotangent crosses it. */
int oc_backward(const oc_config *c, const oc_scene *sc, const double *act, const double *states,
                const double *spre, const uint8_t *done, const int32_t *hit_cam,
                const int32_t *hit_lid, const double *g_r, const double *g_depth,
                const double *g_lidar, const double *g_sT, const double *g_imu,
                const int32_t *gate_tape, double *g_a, double *g_s0, int n_threads)
{
    ctx_t x;
    ctx_init(&x, c, sc);
    int N = c->n_env, M = c->n_agent, T = c->horizon, D = x.D, A = x.A, NM = x.NM;
    memset(g_a, 0, sizeof(double) * (size_t)T * NM * A);
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int env = 0; env < N; ++env) {
        map_t mp;
        map_of(&x, env, &mp);
        int i0 = env * M;
        double *gs = calloc((size_t)M * D, sizeof(double));
        double *gpre = calloc((size_t)M * D, sizeof(double));
        double *gs0x = calloc((size_t)M * D, sizeof(double)); /* direct terms on s_t */
        double drag = sc->drag_env ? sc->drag_env[env] : c->drag;
        if (g_sT) memcpy(gs, g_sT + (size_t)i0 * D, sizeof(double) * M * D);
        for (int t = T - 1; t >= 0; --t) {
            size_t sT = (size_t)t * NM;
            int dn = done[sT + i0];
            /* cotangent of s_{t+1} (after reset) -> before reset */
            for (int m = 0; m < M; ++m) {
                int i = i0 + m;
                double *g = gs + (size_t)m * D;
                if (!dn)
                    render_vjp(&x, env, states + (sT + NM + i) * D,
                               hit_cam + (sT + i) * x.Rc, hit_lid + (sT + i) * x.Rl,
                               g_depth ? g_depth + (sT + i) * x.Rc : NULL,
                               g_lidar ? g_lidar + (sT + i) * x.Rl : NULL, g);
                for (int k = 0; k < D; ++k) gpre[(size_t)m * D + k] = dn ? 0.0 : g[k];
            }
            /* reward on the state before reset */
            for (int m = 0; m < M; ++m) {
                int i = i0 + m, id;
                double gr = g_r[sT + i];
                const double *p = spre + (sT + i) * D;
                const double *a = act + (sT + i) * A;
                double *gp = gpre + (size_t)m * D;
                double *gaa = g_a + (sT + i) * A;
                if (c->task == 1) {
                    /* progress w_pos (|p_t - g| - |p_{t+1} - g|) */
                    const double *g = mp.gate + 7 * gate_tape[sT + i];
                    const double *p0 = states + (sT + i) * D;
                    double e0[3] = {p0[0] - g[0], p0[1] - g[1], p0[2] - g[2]};
                    double e1[3] = {p[0] - g[0], p[1] - g[1], p[2] - g[2]};
                    double n0 = norm3(e0), n1 = norm3(e1);
                    for (int k = 0; k < 3; ++k) {
                        if (n0 > 0.0) gs0x[(size_t)m * D + k] += gr * c->w_pos * e0[k] / n0;
                        if (n1 > 0.0) gp[k] += -gr * c->w_pos * e1[k] / n1;
                    }
                } else {
                    const double *tg = sc->targets + 3 * (size_t)i;
                    double e[3] = {p[0] - tg[0], p[1] - tg[1], p[2] - tg[2]};
                    double ne = norm3(e);
                    for (int k = 0; k < 3; ++k) {
                        double dpos = c->pos_sq ? 2.0 * e[k] : (ne > 0.0 ? e[k] / ne : 0.0);
                        gp[k] += -gr * c->w_pos * dpos;
                    }
                }
                if (g_imu && !dn)
                    imu_vjp(c, drag, states + (sT + i) * D, a, p, g_imu + (sT + i) * 6,
                            gs0x + (size_t)m * D, gp, gaa);
                if (c->w_obs != 0.0) {
                    double gap;
                    double sd = sdf_min(p, &mp, &id, &gap);
                    double ob = sd < OC_INF ? relu(c->d_safe - sd) : 0.0;
                    if (ob > 0.0) {
                        double gsd[3];
                        sdf_grad(p, &mp, id, gsd);
                        for (int k = 0; k < 3; ++k) gp[k] += gr * 2.0 * c->w_obs * ob * gsd[k];
                    }
                }
                for (int k = 0; k < A; ++k) gaa[k] += -2.0 * c->w_act * gr * a[k];
                for (int n = 0; n < M; ++n) {
                    if (n == m) continue;
                    const double *q = spre + (sT + i0 + n) * D;
                    double dd[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
                    double dij = norm3(dd);
                    double sv = relu(c->d_agent - dij);
                    if (sv > 0.0 && dij > 0.0) {
                        /* r_m and r_n both hold -w sv^2; d/dp_m of -w sv^2 = 2 w sv dd/dij */
                        double gsum = gr + g_r[sT + i0 + n];
                        for (int k = 0; k < 3; ++k) gp[k] += gsum * 2.0 * c->w_agent * sv * dd[k] / dij;
                    }
                }
            }
            /* dynamics */
            for (int m = 0; m < M; ++m) {
                int i = i0 + m;
                double *g = gs + (size_t)m * D;
                memset(g, 0, sizeof(double) * D);
                const double *s = states + (sT + i) * D;
                const double *a = act + (sT + i) * A;
                if (c->model == OC_RIGID)
                    rb_step_vjp(c, s, a, gpre + (size_t)m * D, g, g_a + (sT + i) * A);
                else if (c->model == OC_PMD)
                    pmd_step_vjp(c, a, gpre + (size_t)m * D, g, g_a + (sT + i) * A);
                else if (c->model == OC_SIMPLE)
                    simple_step_vjp(c, s, a, gpre + (size_t)m * D, g, g_a + (sT + i) * A);
                else {
                    double lam = sc->lam_env ? sc->lam_env[env] : c->lam;
                    pm_step_vjp(c, drag, lam, s, a, gpre + (size_t)m * D, g, g_a + (sT + i) * A);
                }
                for (int k = 0; k < D; ++k) {
                    g[k] += gs0x[(size_t)m * D + k];
                    gs0x[(size_t)m * D + k] = 0.0;
                }
            }
        }
        memcpy(g_s0 + (size_t)i0 * D, gs, sizeof(double) * M * D);
        free(gs);
        free(gpre);
        free(gs0x);
    }
    ctx_free(&x);
    return 0;
}

/* Scalar loss of a recorded rollout with given cotangents, i.e. the linear
 * functional whose gradient oc_backward returns:
 *   L = sum g_r r_ctrl + sum g_depth depth + sum g_lidar lidar + g_sT . s_T.
 * Used by the finite-difference checks. */
double oc_loss(const oc_config *c, const oc_scene *sc, const double *s0, const double *act,
               const double *g_r, const double *g_depth, const double *g_lidar,
               const double *g_sT, const double *g_imu, const int32_t *gate_k0,
               const double *imu_noise, const double *imu_bias0)
{
    ctx_t x;
    ctx_init(&x, c, sc);
    int N = c->n_env, T = c->horizon, D = x.D, NM = x.NM;
    size_t ns = (size_t)(T + 1) * NM * D;
    double *states = malloc(sizeof(double) * ns);
    double *spre = malloc(sizeof(double) * (size_t)T * NM * D);
    double *r = malloc(sizeof(double) * (size_t)T * NM);
    int8_t *rg = malloc((size_t)T * NM);
    uint8_t *dn = malloc((size_t)T * NM), *as = malloc((size_t)T * NM);
    int32_t *sid = malloc(sizeof(int32_t) * (size_t)T * NM);
    size_t nc = (size_t)T * NM * x.Rc, nl = (size_t)T * NM * x.Rl;
    double *dep = malloc(sizeof(double) * (nc ? nc : 1)), *lid = malloc(sizeof(double) * (nl ? nl : 1));
    int32_t *hc = malloc(sizeof(int32_t) * (nc ? nc : 1)), *hl = malloc(sizeof(int32_t) * (nl ? nl : 1));
    uint8_t *ac = malloc(nc ? nc : 1), *al = malloc(nl ? nl : 1);
    int32_t *pk = calloc((size_t)N, sizeof(int32_t));
    int32_t *gk = calloc((size_t)NM, sizeof(int32_t));
    double *imu = malloc(sizeof(double) * (size_t)T * NM * 6);
    double *bias = calloc((size_t)NM * 6, sizeof(double));
    if (gate_k0) memcpy(gk, gate_k0, sizeof(int32_t) * NM);
    if (imu_bias0) memcpy(bias, imu_bias0, sizeof(double) * NM * 6);
    oc_extra ex = {gk, NULL, imu, imu_noise, bias};
    oc_rollout(c, sc, s0, pk, act, states, spre, r, rg, dn, dep, lid, hc, hl, ac, al, as, sid, &ex, 1);
    double L = 0.0;
    if (g_imu) for (size_t k = 0; k < (size_t)T * NM * 6; ++k) L += g_imu[k] * imu[k];
    for (size_t k = 0; k < (size_t)T * NM; ++k) L += g_r[k] * r[k];
    if (g_depth) for (size_t k = 0; k < nc; ++k) L += g_depth[k] * dep[k];
    if (g_lidar) for (size_t k = 0; k < nl; ++k) L += g_lidar[k] * lid[k];
    if (g_sT) for (size_t k = 0; k < (size_t)NM * D; ++k) L += g_sT[k] * states[(size_t)T * NM * D + k];
    free(states); free(spre); free(r); free(rg); free(dn); free(as); free(sid);
    free(dep); free(lid); free(hc); free(hl); free(ac); free(al); free(pk);
    free(gk); free(imu); free(bias);
    ctx_free(&x);
    return L;
}

/* Largest thread count OpenMP would use (for reporting). */
int oc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
