// sim_kernels.cuh -- kernel argument blocks, shared-memory layout and the
// ray-casting building blocks shared by the rollout and adjoint kernels.
#pragma once
#include "sim_device.cuh"

namespace ds {

constexpr int MAX_SENSORS = 2;

// Hit queues of one warp of the render adjoint: one per group of VL lanes
// (an item each), VQ_CAP entries (ray slot, output cotangent, primitive id);
// VQ_FLUSH blocks of VL rays at most between flushes.
constexpr int VL = 8;
constexpr int VQ_PER_WARP = 32 / VL;
constexpr int VQ_FLUSH = 16;
constexpr int VQ_CAP = VL * VQ_FLUSH;
constexpr int VQ_BYTES = VQ_PER_WARP * VQ_CAP * 10;
static_assert(VQ_FLUSH % 4 == 0, "the taped adjoint gathers rounds of 4 blocks between flushes");

// Capacities of a cull list (the largest per-map counts of each kind).
struct LCap {
    int ns, nb, nc, ng;
};

// One ray sensor: the camera (kind 0, z-depth) or the LiDAR (kind 1, range).
struct Sensor {
    int R;                 // rays per agent
    const float4* dir;     // [R] body-frame unit direction (x, y, z) and output factor w
    const float* tmax;     // [R] ray length at the output clamp (range / w camera, range LiDAR)
    const int* pix;        // [R] output ray index of each table slot (tile order), nullptr: identity
    const float4* cone;    // [chunks] cone of each chunk of 32 x rays-per-thread slots: axis, cos
    const float* cone_sin; // [chunks] sin of the cone's half-angle
    float range;           // output clamp
    int kind;              // 0 camera frustum cull, 1 LiDAR elevation-band cull
    float c0, c1, c2, c3;  // camera: tan_h, tan_v, 1/sqrt(1+tan_h^2), 1/sqrt(1+tan_v^2)
                           // lidar:  elev_lo, elev_hi
    float maxlen;          // longest ray length that is not clamped
    float* out;            // [T][NM][R] output or nullptr
    int16_t* tape;         // [T][NM][R] hit ids or nullptr
    const float* gout;     // adjoint: [T][NM][R] cotangent or nullptr
};

// Byte offsets of the dynamic shared-memory regions of one CTA.
struct Smem {
    int prim;    // float4 [ns_max + 2 (nb_max + nc_max + ng_max)]  map block
    int lsph;    // float4 [L][ns_max]             (oc.xyz, -sqrt(C)) per culled sphere
    int lr2;     // float2 [L][ns_max]             (C, r) per culled sphere
    int lbox;    // float4 [L][nb_max][2]          (centre - o, half extents) per culled box
    int lid;     // short  [L][ns_max + nb_max]    primitive id of each list entry
    int lmeta;   // int4   [L]                     (n_sph, n_box, inside_id, 0)
    int st;      // float  [M][16]                 current state
    int spre;    // float  [M][16]                 state before reset
    int pose;    // float  [M][12]                 o, R
    int aux;     // float  [M][8]                  sdf, collided, g_r, pose cotangent...
    int gpose;   // float  [items][12]             adjoint: per-item pose cotangent partials
    int gs;      // float  [M][16]                 adjoint: state cotangent
    int seg;     // float  [K+1][M][16]            adjoint: segment states
    int mbar;    // uint64 mbarrier
    int wlist;   // render kernels: first per-warp cull list
    int wstride; // render kernels: bytes per warp list
    int vq;      // render adjoint: first per-warp hit queue (VQ_BYTES each)
    int total;
};

struct Args {
    Phys c;
    int N, M, NM, T, K, S;      // envs, agents/env, agents, steps, checkpoint interval, sensors
    int ns_max, nb_max, cull;
    int cast_mode;              // 0 thread per ray, 1 warp per ray (spheres and boxes)
    int nc_max, ng_max;         // largest cylinder and gate counts of a map
    int render_only;            // forward: only render the current state (no dynamics)
    Sensor sen[MAX_SENSORS];
    Smem sm;
    // scene
    const float4* prims; const int* map_off; const int* map_ns; const int* map_nb;
    const int* map_nc; const int* map_ng;   // cylinder and gate counts [n_maps] (nullable: none)
    const int* env_map; const int* order; const float* targets; const float* pool;
    const float* drag_env; const float* lam_env;
    // state and io
    float* state;               // [NM][D] current state (read at start, written at end)
    const float* actions;       // [T][NM][A]
    float* r_ctrl; int8_t* r_goal; uint8_t* done;   // [T][NM] or nullptr
    uint8_t* done_tape;         // [T][NM] internal
    int16_t* sdf_tape;          // [T][NM] internal
    float* ckpt; int* ckpt_k;   // [nseg][NM][D], [nseg][N]
    int* pool_k;                // [N]
    // adjoint
    const float* g_r; const float* g_sT; float* g_a; float* g_s0;
    const uint8_t* done_rd;     // adjoint: [T][NM] done flags of the forward pass
    float* poses;               // [T][NM][12] sensor pose per step (origin, row-major R)
    float* gposes;              // [T][NM][parts][12] cotangent of the poses, per ray part
    int parts;                  // ray parts per (step, agent) item of the render adjoint
    int rparts[MAX_SENSORS];    // forward render: ray parts per (step, agent, sensor) item
    // racing (task 1) and IMU
    int* gate_k;                // [NM] each agent's next gate, read and advanced
    int16_t* gate_tape;         // [T][NM] gate targeted during step t (internal)
    float* imu;                 // [T][NM][6] readout or nullptr
    const float* imu_noise;     // [T][NM][12] standard normal samples or nullptr
    float* imu_bias;            // [NM][6] bias state (advanced with imu_noise)
    const float* g_imu;         // adjoint: [T][NM][6] cotangent of the readout or nullptr
    // control
    int* work; int* status;
    int wait_polls;             // > 0: poll limit of the map copy's wait (tests of the timeout path)
    unsigned long long* counters;  // [4]: sphere tests, box / cylinder / gate tests, rays, env-steps (nullable)
};

__device__ __forceinline__ LCap cap_of(const Args& a) { return LCap{a.ns_max, a.nb_max, a.nc_max, a.ng_max}; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// --------------------------------------------------------- TMA bulk staging
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy `bytes` (multiple of 16, both addresses 16-byte aligned) from global
// to shared memory with one cp.async.bulk completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for the mbarrier phase; false after ~2^22 polls (seconds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    for (int i = 0; i < (1 << 22); ++i) {
        if (mbar_try(bar, phase)) return true;
        if (i > 64) __nanosleep(256);
    }
    return false;
}

// Non-blocking test of the mbarrier phase.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// The first wait of a CTA: polls > 0 limits it to that many non-blocking
// tests (a host-set limit that lets a test make the wait run out); 0 waits
// as mbar_wait does.
__device__ __forceinline__ bool mbar_wait_first(uint64_t* bar, uint32_t phase, int polls) {
    if (polls <= 0) return mbar_wait(bar, phase);
    for (int i = 0; i < polls; ++i)
        if (mbar_test(bar, phase)) return true;
    return false;
}

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ void warp_argmin(float& v, int& id) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, id, o);
        if (v2 < v || (v2 == v && (unsigned)i2 < (unsigned)id)) { v = v2; id = i2; }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- culling
// Conservative test: can any ray of the sensor reach the bounding sphere
// (centre oc relative to the origin, radius rho) before its clamp?  The
// sensor's constants are gathered once per list (CullK), and the camera test
// is evaluated without early exits (one predicate chain, no divergence).
struct CullK {
    float c2, c0c2, c3, c1c3;  // camera: frustum plane factors
    float reach;               // longest unclamped ray + margin
    float lo, hi;              // LiDAR elevation band (with margin)
    int kind;
};

__device__ __forceinline__ CullK cull_consts(const Sensor& s) {
    CullK k;
    k.c2 = s.c2; k.c0c2 = s.c0 * s.c2; k.c3 = s.c3; k.c1c3 = s.c1 * s.c3;
    k.reach = s.maxlen + 1e-3f;
    k.lo = s.c0 - 1e-3f; k.hi = s.c1 + 1e-3f;
    k.kind = s.kind;
    return k;
}

__device__ __forceinline__ bool cull_keep(const CullK& s, const float* R, const float* oc, float rho) {
    const float L2 = dot3(oc, oc), r = rho + 1e-3f, rout = s.reach + rho;
    const bool near = L2 <= r * r;        // |oc| <= rho + m: the origin may be inside
    const bool far = L2 > rout * rout;    // |oc| - rho > maxlen + m: beyond every ray
    // body-frame centre c_B = R^T oc
    const float bx = fmaf(R[0], oc[0], fmaf(R[3], oc[1], R[6] * oc[2]));
    const float by = fmaf(R[1], oc[0], fmaf(R[4], oc[1], R[7] * oc[2]));
    const float bz = fmaf(R[2], oc[0], fmaf(R[5], oc[1], R[8] * oc[2]));
    if (s.kind == 0) {
        // four side planes of the pinhole frustum through the origin: signed
        // distance (tan * x -+ y) / sqrt(1 + tan^2) = (c0 c2) x -+ c2 y
        const float hx = s.c0c2 * bx, vx = s.c1c3 * bx;
        const bool in = (fmaf(-s.c2, by, hx) >= -r) & (fmaf(s.c2, by, hx) >= -r) & (fmaf(-s.c3, bz, vx) >= -r) &
                        (fmaf(s.c3, bz, vx) >= -r);
        return !far & in;  // |oc| <= r passes every plane through the origin
    }
    if (near) return true;
    if (far) return false;
    const float L = sqrtf(L2);
    const float el = asinf(fminf(fmaxf(bz / L, -1.f), 1.f));
    const float del = asinf(fminf(r / L, 1.f));
    return (el - del <= s.hi) && (el + del >= s.lo);
}

}  // namespace ds
