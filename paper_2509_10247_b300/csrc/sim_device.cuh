// sim_device.cuh -- per-agent FP32 device math of the fused quadrotor step:
// dynamics (Eq. 1, Eq. 2, Eq. 3, Eq. 4), sensor pose (Sec. III-B), signed distances,
// rewards (Sec. III-C/D/E) and their vector-Jacobian products (Eq. 5).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace ds {

enum { MODEL_PM = 0, MODEL_RIGID = 1, MODEL_PMD = 2, MODEL_SIMPLE = 3 };

// Physics and task constants (kernel-parameter resident).
struct Phys {
    int model, M, D, A;
    float dt, g, lam, drag, act_scale, ema_alpha;
    float mass, J[3], K[3], Dd[3], rs[3];
    int pos_sq;
    float w_pos, w_obs, d_safe, w_act, w_agent, d_agent, success_radius, r_quad;
    float blo[3], bhi[3];
    int terminate, P;
    int task;                  // 0 reach / avoid, 1 racing through the map's gates
    float imu_noise[2], imu_walk[2];  // IMU white-noise and bias-walk std (force, rate)
};

// Square root by the hardware approximation (relative error about 2^-22,
// exact at 0): distances and ray-sphere near roots need no correct rounding
// (an error of ~1e-7 of the value is far inside every tolerance).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float clip1(float x) { return fminf(fmaxf(x, -1.f), 1.f); }
__device__ __forceinline__ float dclip1(float x) { return (x >= -1.f && x <= 1.f) ? 1.f : 0.f; }
__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }
__device__ __forceinline__ float dot3(const float* a, const float* b) {
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}
__device__ __forceinline__ void cross3(const float* a, const float* b, float* o) {
    float x = a[1] * b[2] - a[2] * b[1];
    float y = a[2] * b[0] - a[0] * b[2];
    float z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}

// Row-major rotation body -> world of the Hamilton quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(const float* q, float* R) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// d<R(q), G>/dq for row-major G: partial derivatives of the polynomial R(q).
__device__ __forceinline__ void quat_rot_vjp(const float* q, const float* G, float* gq) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    // d/dw: 2 [0 -z y; z 0 -x; -y x 0]
    gq[0] += 2.f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
    // d/dx: 2 [0 y z; y -2x -w; z w -2x]
    gq[1] += 2.f * (y * G[1] + z * G[2] + y * G[3] - 2.f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.f * x * G[8]);
    // d/dy: 2 [-2y x w; x 0 z; -w z -2y]
    gq[2] += 2.f * (-2.f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.f * y * G[8]);
    // d/dz: 2 [-2z -w x; w -2z y; x y 0]
    gq[3] += 2.f * (-2.f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

// ------------------------------------------------------------------ dynamics
// Eq. 3, explicit Euler; the velocity EMA feeds the point-mass heading.
__device__ __forceinline__ void pm_step(const Phys& c, float drag, float lam, const float* s,
                                        const float* act, float* o) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float u = c.act_scale * clip1(act[i]);
        float gi = (i == 2) ? -c.g : 0.f;
        float p = s[i], v = s[3 + i], a = s[6 + i], e = s[9 + i];
        float vn = v + c.dt * (a + gi - drag * v);
        o[i] = p + c.dt * v;
        o[3 + i] = vn;
        o[6 + i] = a + c.dt * lam * (u - a);
        o[9 + i] = (1.f - c.ema_alpha) * e + c.ema_alpha * vn;
    }
}

// Eq. 4, discrete point mass: p' = p + v dt + (u + g) dt^2 / 2,
// v' = v + ((u + g) + (u' + g)) dt / 2, where the state's acceleration slot
// holds the command in force u and the action gives the next one u'.
__device__ __forceinline__ void pmd_step(const Phys& c, const float* s, const float* act, float* o) {
    const float dt = c.dt;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float gi = (i == 2) ? -c.g : 0.f;
        const float p = s[i], v = s[3 + i], u = s[6 + i], e = s[9 + i];
        const float u1 = c.act_scale * clip1(act[i]);
        const float vn = v + 0.5f * ((u + gi) + (u1 + gi)) * dt;
        o[i] = p + v * dt + 0.5f * (u + gi) * dt * dt;
        o[3 + i] = vn;
        o[6 + i] = u1;
        o[9 + i] = (1.f - c.ema_alpha) * e + c.ema_alpha * vn;
    }
}

__device__ __forceinline__ void pmd_step_vjp(const Phys& c, const float* act, const float* go, float* gs,
                                             float* ga) {
    const float al = c.ema_alpha, dt = c.dt;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float gp = go[i], gv = go[3 + i] + al * go[9 + i];
        gs[9 + i] += (1.f - al) * go[9 + i];
        gs[i] += gp;
        gs[3 + i] += dt * gp + gv;
        gs[6 + i] += 0.5f * dt * dt * gp + 0.5f * dt * gv;
        ga[i] += c.act_scale * dclip1(act[i]) * (go[6 + i] + 0.5f * dt * gv);
    }
}

// Eq. 2, simplified quadrotor: state (p, v, R row-major), thrust
// acceleration c = g (1 + clip(a0)) along z_B, body rates omega = rate_scale
// clip(a1..3) as inputs; explicit Euler R~ = R (I + dt [omega]_x), then
// Gram-Schmidt on the columns (x, y orthogonalised, z = x cross y).
__device__ __forceinline__ void simple_pre(const Phys& c, const float* s, const float* act, float* Rt, float* w,
                                           float& cth) {
    const float* R = s + 6;
    cth = c.g * (1.f + clip1(act[0]));
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = c.rs[i] * clip1(act[1 + i]);
    const float W[9] = {0.f, -w[2], w[1], w[2], 0.f, -w[0], -w[1], w[0], 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float acc = R[3 * i] * W[j] + R[3 * i + 1] * W[3 + j] + R[3 * i + 2] * W[6 + j];
            Rt[3 * i + j] = R[3 * i + j] + c.dt * acc;
        }
}

struct GsFrame {
    float x[3], y[3], u1[3], n0, n1, sx;
};

__device__ __forceinline__ void gram_schmidt(const float* Rt, GsFrame& f) {
    const float u0[3] = {Rt[0], Rt[3], Rt[6]};
    f.u1[0] = Rt[1]; f.u1[1] = Rt[4]; f.u1[2] = Rt[7];
    f.n0 = sqrtf(dot3(u0, u0));
#pragma unroll
    for (int i = 0; i < 3; ++i) f.x[i] = u0[i] / f.n0;
    f.sx = dot3(f.x, f.u1);
    float wv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) wv[i] = f.u1[i] - f.sx * f.x[i];
    f.n1 = sqrtf(dot3(wv, wv));
#pragma unroll
    for (int i = 0; i < 3; ++i) f.y[i] = wv[i] / f.n1;
}

__device__ __forceinline__ void simple_step(const Phys& c, const float* s, const float* act, float* o) {
    float Rt[9], w[3], cth;
    simple_pre(c, s, act, Rt, w, cth);
    const float* R = s + 6;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float gi = (i == 2) ? -c.g : 0.f;
        o[i] = s[i] + c.dt * s[3 + i];
        o[3 + i] = s[3 + i] + c.dt * (R[3 * i + 2] * cth + gi);
    }
    GsFrame f;
    gram_schmidt(Rt, f);
    float z[3];
    cross3(f.x, f.y, z);
#pragma unroll
    for (int i = 0; i < 3; ++i) { o[6 + 3 * i] = f.x[i]; o[7 + 3 * i] = f.y[i]; o[8 + 3 * i] = z[i]; }
}

__device__ __forceinline__ void simple_step_vjp(const Phys& c, const float* s, const float* act, const float* go,
                                                float* gs, float* ga) {
    float Rt[9], w[3], cth;
    simple_pre(c, s, act, Rt, w, cth);
    const float* R = s + 6;
    const float dt = c.dt;
    float gc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gs[i] += go[i];
        gs[3 + i] += dt * go[i] + go[3 + i];
        gs[6 + 3 * i + 2] += dt * cth * go[3 + i];
        gc += dt * R[3 * i + 2] * go[3 + i];
    }
    GsFrame f;
    gram_schmidt(Rt, f);
    const float* gRo = go + 6;
    float gx[3] = {gRo[0], gRo[3], gRo[6]}, gy[3] = {gRo[1], gRo[4], gRo[7]}, gz[3] = {gRo[2], gRo[5], gRo[8]};
    float t[3];
    cross3(f.y, gz, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) gx[i] += t[i];
    cross3(gz, f.x, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) gy[i] += t[i];
    const float yg = dot3(f.y, gy);
    float gw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) gw[i] = (gy[i] - f.y[i] * yg) / f.n1;
    const float xg = dot3(f.x, gw);
    float gRt[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gRt[3 * i + 1] = gw[i] - f.x[i] * xg;
        gx[i] -= xg * f.u1[i] + f.sx * gw[i];
    }
    const float xx = dot3(f.x, gx);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gRt[3 * i] = (gx[i] - f.x[i] * xx) / f.n0;
        gRt[3 * i + 2] = 0.f;
    }
    const float W[9] = {0.f, -w[2], w[1], w[2], 0.f, -w[0], -w[1], w[0], 0.f};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float acc = gRt[3 * i] * W[3 * j] + gRt[3 * i + 1] * W[3 * j + 1] + gRt[3 * i + 2] * W[3 * j + 2];
            gs[6 + 3 * i + j] += gRt[3 * i + j] + dt * acc;
        }
    float Mt[9];  // R^T gRt
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int b = 0; b < 3; ++b) Mt[3 * a2 + b] = R[a2] * gRt[b] + R[3 + a2] * gRt[3 + b] + R[6 + a2] * gRt[6 + b];
    const float gwr[3] = {dt * (Mt[7] - Mt[5]), dt * (Mt[2] - Mt[6]), dt * (Mt[3] - Mt[1])};
    ga[0] += c.g * dclip1(act[0]) * gc;
#pragma unroll
    for (int i = 0; i < 3; ++i) ga[1 + i] += c.rs[i] * dclip1(act[1 + i]) * gwr[i];
}

// Eq. 1 with the body-rate controller, explicit Euler, quaternion renormalised.
__device__ __forceinline__ void rb_step(const Phys& c, const float* s, const float* act, float* o) {
    const float* q = s + 3; const float* v = s + 7; const float* w = s + 10;
    float T = c.mass * c.g * (1.f + clip1(act[0]));
    float Jw[3], gy[3], wd[3], R[9], vb[3], vd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Jw[i] = c.J[i] * w[i];
    cross3(w, Jw, gy);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float wc = c.rs[i] * clip1(act[1 + i]);
        float tau = c.J[i] * c.K[i] * (wc - w[i]) + gy[i];
        wd[i] = (tau - gy[i]) / c.J[i];
    }
    quat_rot(q, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) vb[j] = c.Dd[j] * (R[j] * v[0] + R[3 + j] * v[1] + R[6 + j] * v[2]);
    float Tm = T / c.mass;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float gi = (i == 2) ? -c.g : 0.f;
        vd[i] = gi + Tm * R[3 * i + 2] - (R[3 * i] * vb[0] + R[3 * i + 1] * vb[1] + R[3 * i + 2] * vb[2]);
    }
    // q (x) (0, w)
    float qd0 = -(q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
    float qd1 = q[0] * w[0] + q[2] * w[2] - q[3] * w[1];
    float qd2 = q[0] * w[1] + q[3] * w[0] - q[1] * w[2];
    float qd3 = q[0] * w[2] + q[1] * w[1] - q[2] * w[0];
    float h = 0.5f * c.dt;
    float qt0 = q[0] + h * qd0, qt1 = q[1] + h * qd1, qt2 = q[2] + h * qd2, qt3 = q[3] + h * qd3;
    float inv = rsqrtf(qt0 * qt0 + qt1 * qt1 + qt2 * qt2 + qt3 * qt3);
    float n[13];
#pragma unroll
    for (int i = 0; i < 3; ++i) n[i] = s[i] + c.dt * v[i];
    n[3] = qt0 * inv; n[4] = qt1 * inv; n[5] = qt2 * inv; n[6] = qt3 * inv;
#pragma unroll
    for (int i = 0; i < 3; ++i) n[7 + i] = v[i] + c.dt * vd[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) n[10 + i] = w[i] + c.dt * wd[i];
#pragma unroll
    for (int i = 0; i < 13; ++i) o[i] = n[i];
}

// Point-mass heading frame (Sec. III-B): z along thrust, x along the
// horizontal velocity EMA made orthogonal to z, y = z x x.
struct PmFrame {
    float z[3], h[3], hp[3], x[3], na, nh, hz;
    bool zfb, hfb;
};

__device__ __forceinline__ void pm_frame(const float* s, PmFrame& f) {
    const float* a = s + 6; const float* e = s + 9;
    f.na = sqrtf(dot3(a, a));
    f.zfb = f.na < 1e-6f;
    if (f.zfb) { f.z[0] = 0.f; f.z[1] = 0.f; f.z[2] = 1.f; }
    else { float r = 1.f / f.na; f.z[0] = a[0] * r; f.z[1] = a[1] * r; f.z[2] = a[2] * r; }
    f.h[0] = e[0]; f.h[1] = e[1]; f.h[2] = 0.f;
    f.hfb = false;
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
        f.hz = dot3(f.h, f.z);
#pragma unroll
        for (int i = 0; i < 3; ++i) f.hp[i] = f.h[i] - f.hz * f.z[i];
        f.nh = sqrtf(dot3(f.hp, f.hp));
        if (f.nh >= 1e-6f || k == 2) break;
        f.hfb = true;  // fall back to world +x, then +y
        f.h[0] = (k == 0) ? 1.f : 0.f; f.h[1] = (k == 0) ? 0.f : 1.f; f.h[2] = 0.f;
    }
    float r = 1.f / f.nh;
#pragma unroll
    for (int i = 0; i < 3; ++i) f.x[i] = f.hp[i] * r;
}

// Sensor pose: o = position, R (row-major) = body -> world.
__device__ __forceinline__ void sensor_pose(int model, const float* s, float* o, float* R) {
    o[0] = s[0]; o[1] = s[1]; o[2] = s[2];
    if (model == MODEL_RIGID) { quat_rot(s + 3, R); return; }
    if (model == MODEL_SIMPLE) {
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = s[6 + k];
        return;
    }
    PmFrame f;
    pm_frame(s, f);
    float y[3];
    cross3(f.z, f.x, y);
#pragma unroll
    for (int i = 0; i < 3; ++i) { R[3 * i] = f.x[i]; R[3 * i + 1] = y[i]; R[3 * i + 2] = f.z[i]; }
}

// VJP of the pose: cotangents go (origin) and gR (row-major R) into gs.
__device__ __forceinline__ void pose_vjp(int model, const float* s, const float* go, const float* gR,
                                         float* gs) {
    gs[0] += go[0]; gs[1] += go[1]; gs[2] += go[2];
    if (model == MODEL_RIGID) { quat_rot_vjp(s + 3, gR, gs + 3); return; }
    if (model == MODEL_SIMPLE) {
#pragma unroll
        for (int k = 0; k < 9; ++k) gs[6 + k] += gR[k];
        return;
    }
    PmFrame f;
    pm_frame(s, f);
    float gx[3] = {gR[0], gR[3], gR[6]}, gy[3] = {gR[1], gR[4], gR[7]}, gz[3] = {gR[2], gR[5], gR[8]};
    float t[3];
    cross3(f.x, gy, t);  // y = z x x
    gz[0] += t[0]; gz[1] += t[1]; gz[2] += t[2];
    cross3(gy, f.z, t);
    gx[0] += t[0]; gx[1] += t[1]; gx[2] += t[2];
    float xg = dot3(f.x, gx), ghp[3];
    float rn = 1.f / f.nh;
#pragma unroll
    for (int i = 0; i < 3; ++i) ghp[i] = (gx[i] - f.x[i] * xg) * rn;
    float zg = dot3(f.z, ghp);
#pragma unroll
    for (int i = 0; i < 3; ++i) gz[i] += -f.hz * ghp[i] - f.h[i] * zg;
    if (!f.hfb) { gs[9] += ghp[0] - f.z[0] * zg; gs[10] += ghp[1] - f.z[1] * zg; }
    if (!f.zfb) {
        float zz = dot3(f.z, gz), ra = 1.f / f.na;
#pragma unroll
        for (int i = 0; i < 3; ++i) gs[6 + i] += (gz[i] - f.z[i] * zz) * ra;
    }
}

// VJP of the point-mass step.
__device__ __forceinline__ void pm_step_vjp(const Phys& c, float drag, float lam, const float* act,
                                            const float* go, float* gs, float* ga) {
    float al = c.ema_alpha, dt = c.dt;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float gp = go[i], gv = go[3 + i] + al * go[9 + i], gA = go[6 + i];
        gs[9 + i] += (1.f - al) * go[9 + i];
        gs[i] += gp;
        gs[3 + i] += dt * gp + (1.f - dt * drag) * gv;
        gs[6 + i] += dt * gv + (1.f - dt * lam) * gA;
        ga[i] += c.act_scale * dclip1(act[i]) * (dt * lam * gA);
    }
}

// VJP of the rigid-body step (recomputes the forward intermediates).
__device__ __forceinline__ void rb_step_vjp(const Phys& c, const float* s, const float* act,
                                            const float* go, float* gs, float* ga) {
    const float* q = s + 3; const float* v = s + 7; const float* w = s + 10;
    float dt = c.dt, m = c.mass;
    float T = m * c.g * (1.f + clip1(act[0]));
    float R[9], dvb[3], Jw[3];
    quat_rot(q, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) dvb[j] = c.Dd[j] * (R[j] * v[0] + R[3 + j] * v[1] + R[6 + j] * v[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) Jw[i] = c.J[i] * w[i];
    float qd0 = -(q[1] * w[0] + q[2] * w[1] + q[3] * w[2]);
    float qd1 = q[0] * w[0] + q[2] * w[2] - q[3] * w[1];
    float qd2 = q[0] * w[1] + q[3] * w[0] - q[1] * w[2];
    float qd3 = q[0] * w[2] + q[1] * w[1] - q[2] * w[0];
    float h = 0.5f * dt;
    float qt[4] = {q[0] + h * qd0, q[1] + h * qd1, q[2] + h * qd2, q[3] + h * qd3};
    float nq = sqrtf(qt[0] * qt[0] + qt[1] * qt[1] + qt[2] * qt[2] + qt[3] * qt[3]);
    float rq = 1.f / nq;
    float qn[4] = {qt[0] * rq, qt[1] * rq, qt[2] * rq, qt[3] * rq};

    const float* gqn = go + 3; const float* gvn = go + 7; const float* gwn = go + 10;
    float gvd[3], gwd[3], gqd[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gs[i] += go[i];
        gs[7 + i] += dt * go[i] + gvn[i];
        gvd[i] = dt * gvn[i];
        gs[10 + i] += gwn[i];
        gwd[i] = dt * gwn[i];
    }
    float qg = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float gqt = (gqn[k] - qn[k] * qg) * rq;
        gs[3 + k] += gqt;
        gqd[k] = h * gqt;
    }
    // qd = q (x) (0, w)
    {
        float vq[3] = {q[1], q[2], q[3]}, gv3[3] = {gqd[1], gqd[2], gqd[3]}, t[3];
        gs[3] += dot3(gv3, w);
        cross3(w, gv3, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) gs[4 + i] += -gqd[0] * w[i] + t[i];
        cross3(gv3, vq, t);
#pragma unroll
        for (int i = 0; i < 3; ++i) gs[10 + i] += -gqd[0] * vq[i] + q[0] * gv3[i] + t[i];
    }
    // vd = g + (T/m) R e3 - R dvb,  dvb = D (R^T v)
    float gR[9], gT = 0.f, gvb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gT += R[3 * i + 2] * gvd[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) gR[3 * i + j] = -gvd[i] * dvb[j];
        gR[3 * i + 2] += (T / m) * gvd[i];
    }
    gT /= m;
#pragma unroll
    for (int j = 0; j < 3; ++j) gvb[j] = -c.Dd[j] * (R[j] * gvd[0] + R[3 + j] * gvd[1] + R[6 + j] * gvd[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gs[7 + i] += R[3 * i] * gvb[0] + R[3 * i + 1] * gvb[1] + R[3 * i + 2] * gvb[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) gR[3 * i + j] += v[i] * gvb[j];
    }
    quat_rot_vjp(q, gR, gs + 3);
    // wd = (tau - gy)/J, tau = J K (wc - w) + gy, gy = w x Jw
    float gtau[3], ggy[3], t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gtau[i] = gwd[i] / c.J[i];
        ggy[i] = -gtau[i] + gtau[i];
        gs[10 + i] += -c.J[i] * c.K[i] * gtau[i];
        ga[1 + i] += c.rs[i] * dclip1(act[1 + i]) * (c.J[i] * c.K[i] * gtau[i]);
    }
    cross3(Jw, ggy, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) gs[10 + i] += t[i];
    cross3(ggy, w, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) gs[10 + i] += c.J[i] * t[i];
    ga[0] += m * c.g * dclip1(act[0]) * gT;
}

// ---------------------------------------------------------------- obstacles
// Map block in memory (float4): ns spheres (cx, cy, cz, r); nb boxes as
// (min xyz, 0), (max xyz, 0); nc vertical capped cylinders as (cx, cy, r, 0),
// (zmin, zmax, 0, 0); ng racing gates as (cx, cy, cz, w), (cos yaw, sin yaw,
// b, hd).  Primitive ids: spheres 0.., boxes ns.., cylinders ns + nb..,
// gates ns + nb + nc...
struct MapView {
    const float4* prim;
    int ns, nb, nc, ng;
    __device__ __forceinline__ int count() const { return ns + nb + nc + ng; }
    __device__ __forceinline__ const float4* box(int k) const { return prim + ns + 2 * k; }
    __device__ __forceinline__ const float4* cyl(int k) const { return prim + ns + 2 * nb + 2 * k; }
    __device__ __forceinline__ const float4* gate(int k) const { return prim + ns + 2 * (nb + nc) + 2 * k; }
};

// Local gate coordinates (normal, lateral, up) of a point relative to the centre.
__device__ __forceinline__ void gate_local(const float4& g0, const float4& g1, const float* p, float* u) {
    const float rx = p[0] - g0.x, ry = p[1] - g0.y;
    u[0] = fmaf(g1.x, rx, g1.y * ry);
    u[1] = fmaf(g1.x, ry, -g1.y * rx);
    u[2] = p[2] - g0.z;
}

// Signed distance of a box given by centre ctr and half extents h (local frame).
__device__ __forceinline__ float sdf_box_ch(const float* q0, const float* ctr, const float* h) {
    float q[3], out = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        q[i] = fabsf(q0[i] - ctr[i]) - h[i];
        out = fmaf(relu(q[i]), relu(q[i]), out);
    }
    return sqrt_approx(out) + fminf(fmaxf(q[0], fmaxf(q[1], q[2])), 0.f);
}

// Bar k of a gate (0 top, 1 bottom, 2 left, 3 right) in local coordinates:
// centre and half extents; top and bottom span the outer width, the sides
// the opening's height.
__device__ __forceinline__ void gate_bar(const float4& g0, const float4& g1, int k, float* ctr, float* h) {
    const float w = g0.w, b = g1.z, m = w + 0.5f * b;
    ctr[0] = 0.f;
    h[0] = g1.w;
    ctr[1] = k < 2 ? 0.f : (k == 2 ? -m : m);
    ctr[2] = k < 2 ? (k == 0 ? m : -m) : 0.f;
    h[1] = k < 2 ? w + b : 0.5f * b;
    h[2] = k < 2 ? 0.5f * b : w;
}

__device__ __forceinline__ float sdf_gate(const float4& g0, const float4& g1, const float* p, int* bar) {
    float u[3];
    gate_local(g0, g1, p, u);
    float best = CUDART_INF_F;
    int bi = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float ctr[3], h[3];
        gate_bar(g0, g1, k, ctr, h);
        const float d = sdf_box_ch(u, ctr, h);
        if (d < best) { best = d; bi = k; }
    }
    *bar = bi;
    return best;
}

// Signed distance of p to a sphere (c, r).
__device__ __forceinline__ float sdf_sphere(const float4& s, const float* p) {
    const float dx = p[0] - s.x, dy = p[1] - s.y, dz = p[2] - s.z;
    return sqrt_approx(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - s.w;
}

// Signed distance of p to an axis-aligned box given by its corners.
__device__ __forceinline__ float sdf_box_lohi(const float4& lo, const float4& hi, const float* p) {
    const float qx = fabsf(p[0] - 0.5f * (lo.x + hi.x)) - 0.5f * (hi.x - lo.x);
    const float qy = fabsf(p[1] - 0.5f * (lo.y + hi.y)) - 0.5f * (hi.y - lo.y);
    const float qz = fabsf(p[2] - 0.5f * (lo.z + hi.z)) - 0.5f * (hi.z - lo.z);
    const float ox = relu(qx), oy = relu(qy), oz = relu(qz);
    const float in = fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
    return sqrt_approx(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) + in;
}

__device__ __forceinline__ float sdf_prim(const MapView& m, int k, const float* p) {
    if (k < m.ns) return sdf_sphere(m.prim[k], p);
    k -= m.ns;
    if (k < m.nb) return sdf_box_lohi(m.box(k)[0], m.box(k)[1], p);
    k -= m.nb;
    if (k < m.nc) {
        const float4 c0 = m.cyl(k)[0], c1 = m.cyl(k)[1];
        const float ex = p[0] - c0.x, ey = p[1] - c0.y;
        const float qr = sqrt_approx(fmaf(ex, ex, ey * ey)) - c0.z;
        const float qz = fabsf(p[2] - 0.5f * (c1.x + c1.y)) - 0.5f * (c1.y - c1.x);
        return sqrt_approx(fmaf(relu(qr), relu(qr), relu(qz) * relu(qz))) + fminf(fmaxf(qr, qz), 0.f);
    }
    k -= m.nc;
    int bar;
    return sdf_gate(m.gate(k)[0], m.gate(k)[1], p, &bar);
}

// Gradient of a box's signed distance (centre / half-extent form).
__device__ __forceinline__ void sdf_box_grad_ch(const float* p, const float* ctr, const float* h, float* gp) {
    float q[3], sg[3], out = 0.f;
    int am = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        sg[i] = (p[i] - ctr[i] >= 0.f) ? 1.f : -1.f;
        q[i] = fabsf(p[i] - ctr[i]) - h[i];
        out += relu(q[i]) * relu(q[i]);
    }
    if (q[1] > q[am]) am = 1;
    if (q[2] > q[am]) am = 2;
    if (out > 0.f) {
        float r = rsqrtf(out);
#pragma unroll
        for (int i = 0; i < 3; ++i) gp[i] = relu(q[i]) * sg[i] * r;
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) gp[i] = (i == am) ? sg[i] : 0.f;
    }
}

__device__ __forceinline__ void sdf_prim_grad(const MapView& m, int k, const float* p, float* gp) {
    if (k < m.ns) {
        float4 s = m.prim[k];
        float d[3] = {p[0] - s.x, p[1] - s.y, p[2] - s.z};
        float n = sqrtf(dot3(d, d));
        float r = n > 0.f ? 1.f / n : 0.f;
        gp[0] = d[0] * r; gp[1] = d[1] * r; gp[2] = d[2] * r;
        return;
    }
    k -= m.ns;
    if (k < m.nb) {
        float4 lo = m.box(k)[0], hi = m.box(k)[1];
        const float ctr[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
        const float h[3] = {0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z)};
        sdf_box_grad_ch(p, ctr, h, gp);
        return;
    }
    k -= m.nb;
    if (k < m.nc) {
        const float4 c0 = m.cyl(k)[0], c1 = m.cyl(k)[1];
        const float ex = p[0] - c0.x, ey = p[1] - c0.y, zc = 0.5f * (c1.x + c1.y);
        const float rho = sqrtf(fmaf(ex, ex, ey * ey));
        const float qr = rho - c0.z, qz = fabsf(p[2] - zc) - 0.5f * (c1.y - c1.x);
        const float ir = rho > 0.f ? 1.f / rho : 0.f;
        const float sz = p[2] - zc >= 0.f ? 1.f : -1.f;
        const float out = sqrtf(fmaf(relu(qr), relu(qr), relu(qz) * relu(qz)));
        if (out > 0.f) {
            const float io = 1.f / out;
            gp[0] = relu(qr) * ex * ir * io; gp[1] = relu(qr) * ey * ir * io; gp[2] = relu(qz) * sz * io;
        } else if (qr >= qz) {
            gp[0] = ex * ir; gp[1] = ey * ir; gp[2] = 0.f;
        } else {
            gp[0] = 0.f; gp[1] = 0.f; gp[2] = sz;
        }
        return;
    }
    k -= m.nc;
    const float4 g0 = m.gate(k)[0], g1 = m.gate(k)[1];
    int bar;
    sdf_gate(g0, g1, p, &bar);
    float u[3], ctr[3], h[3], gu[3];
    gate_local(g0, g1, p, u);
    gate_bar(g0, g1, bar, ctr, h);
    sdf_box_grad_ch(u, ctr, h, gu);
    gp[0] = fmaf(g1.x, gu[0], -g1.y * gu[1]);
    gp[1] = fmaf(g1.y, gu[0], g1.x * gu[1]);
    gp[2] = gu[2];
}

// Racing: true when the segment x0 -> x1 crosses the gate's centre plane
// from its back (u_n < 0) to its front (u_n >= 0) inside the opening.
__device__ __forceinline__ bool gate_passed(const float4& g0, const float4& g1, const float* x0, const float* x1) {
    float u0[3], u1[3];
    gate_local(g0, g1, x0, u0);
    gate_local(g0, g1, x1, u1);
    if (!(u0[0] < 0.f && u1[0] >= 0.f)) return false;
    const float f = -u0[0] / (u1[0] - u0[0]);
    const float ul = fmaf(f, u1[1] - u0[1], u0[1]), uz = fmaf(f, u1[2] - u0[2], u0[2]);
    return fabsf(ul) < g0.w && fabsf(uz) < g0.w;
}

// ------------------------------------------------------------------- IMU
// Readout of one agent after a step (Sec. III-B), noise-free: specific
// force f = R^T (v' - g) of the model's translational dynamics and the body
// angular rate, in the body frame of the new state s1, the step's action
// held: rigid f = (T/m) e3 - D R^T v, omega from the state; point mass
// f = R^T (a - d v); discrete f = R^T u; simplified f = c e3 and the
// commanded rates; the point-mass rate is the attitude change over the step,
// vee(A - A^T) / (2 dt) with A = R0^T R1.
__device__ __forceinline__ void imu_eval(const Phys& c, float drag, const float* s0, const float* act,
                                         const float* s1, float* out) {
    float o[3], R1[9];
    sensor_pose(c.model, s1, o, R1);
    if (c.model == MODEL_RIGID) {
        const float T = c.g * (1.f + clip1(act[0]));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float vb = fmaf(R1[j], s1[7], fmaf(R1[3 + j], s1[8], R1[6 + j] * s1[9]));
            out[j] = (j == 2 ? T : 0.f) - c.Dd[j] * vb;
            out[3 + j] = s1[10 + j];
        }
        return;
    }
    if (c.model == MODEL_SIMPLE) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            out[j] = j == 2 ? c.g * (1.f + clip1(act[0])) : 0.f;
            out[3 + j] = c.rs[j] * clip1(act[1 + j]);
        }
        return;
    }
    float acc[3], R0[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = c.model == MODEL_PMD ? s1[6 + i] : fmaf(-drag, s1[3 + i], s1[6 + i]);
#pragma unroll
    for (int j = 0; j < 3; ++j) out[j] = fmaf(R1[j], acc[0], fmaf(R1[3 + j], acc[1], R1[6 + j] * acc[2]));
    sensor_pose(c.model, s0, o, R0);
    // A_ij = sum_k R0_ki R1_kj, only the off-diagonal pairs are needed
    auto A = [&](int i, int j) { return fmaf(R0[i], R1[j], fmaf(R0[3 + i], R1[3 + j], R0[6 + i] * R1[6 + j])); };
    const float h = 0.5f / c.dt;
    out[3] = (A(2, 1) - A(1, 2)) * h;
    out[4] = (A(0, 2) - A(2, 0)) * h;
    out[5] = (A(1, 0) - A(0, 1)) * h;
}

// After a reset: the new state read as held at rest (f = -R^T g; the rigid
// body's rate state, else no rate).
__device__ __forceinline__ void imu_reset(const Phys& c, const float* s, float* out) {
    float o[3], R[9];
    sensor_pose(c.model, s, o, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        out[j] = R[6 + j] * c.g;
        out[3 + j] = c.model == MODEL_RIGID ? s[10 + j] : 0.f;
    }
}

// VJP of imu_eval: g [6] into gs0 (state the step started from), gs1 (new
// state before reset) and ga (raw action).
__device__ __forceinline__ void imu_vjp(const Phys& c, float drag, const float* s0, const float* act,
                                        const float* s1, const float* g, float* gs0, float* gs1, float* ga) {
    float o[3], R1[9], gR1[9];
    const float zero[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 9; ++k) gR1[k] = 0.f;
    sensor_pose(c.model, s1, o, R1);
    if (c.model == MODEL_RIGID) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                gR1[3 * i + j] += -c.Dd[j] * s1[7 + i] * g[j];
                gs1[7 + i] += -c.Dd[j] * R1[3 * i + j] * g[j];
            }
        ga[0] += c.g * dclip1(act[0]) * g[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) gs1[10 + j] += g[3 + j];
        pose_vjp(c.model, s1, zero, gR1, gs1);
        return;
    }
    if (c.model == MODEL_SIMPLE) {
        ga[0] += c.g * dclip1(act[0]) * g[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) ga[1 + j] += c.rs[j] * dclip1(act[1 + j]) * g[3 + j];
        return;
    }
    float acc[3], gacc[3] = {0.f, 0.f, 0.f}, R0[9], gR0[9], gA[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { gR0[k] = 0.f; gA[k] = 0.f; }
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = c.model == MODEL_PMD ? s1[6 + i] : fmaf(-drag, s1[3 + i], s1[6 + i]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gR1[3 * i + j] += acc[i] * g[j];
            gacc[i] += R1[3 * i + j] * g[j];
        }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        gs1[6 + i] += gacc[i];
        if (c.model != MODEL_PMD) gs1[3 + i] += -drag * gacc[i];
    }
    sensor_pose(c.model, s0, o, R0);
    const float h = 0.5f / c.dt;
    gA[7] += h * g[3]; gA[5] -= h * g[3];
    gA[2] += h * g[4]; gA[6] -= h * g[4];
    gA[3] += h * g[5]; gA[1] -= h * g[5];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gR0[3 * k + i] += gA[3 * i + j] * R1[3 * k + j];
                gR1[3 * k + j] += gA[3 * i + j] * R0[3 * k + i];
            }
    pose_vjp(c.model, s1, zero, gR1, gs1);
    pose_vjp(c.model, s0, zero, gR0, gs0);
}

}  // namespace ds
