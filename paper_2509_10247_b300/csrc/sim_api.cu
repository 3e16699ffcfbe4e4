// sim_api.cu -- C ABI (include/diffsim.h): handle, validation, scene layout,
// launch-shape selection and the entry points of the fused step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "diffsim.h"
#include "sim_raycast.cuh"

namespace ds {
bool rpt_supported(int rpt);
cudaError_t launch_physics(const Args& a, cudaStream_t st);
cudaError_t launch_physics_bwd(const Args& a, cudaStream_t st);
void physics_bwd_shape(int K, int M, int* warps, size_t* smem);
cudaError_t render_call(bool vjp, bool launch, int rpt, const Args& a, int grid, int block, size_t smem,
                        cudaStream_t st, int* occ);
cudaError_t launch_render_hits(const Args& a, int grid, cudaStream_t st);
}  // namespace ds

using ds::Args;

struct sim_graph;

struct sim_handle {
    sim_config cfg;
    int D = 0, A = 0, N = 0, M = 0, NM = 0, T = 0, K = 0, S = 0, Rc = 0, Rl = 0;
    int device = 0, num_sms = 0;
    bool tape = false;
    // scene
    bool have_scene = false, have_pool = false;
    float4* d_prims = nullptr;
    int *d_map_off = nullptr, *d_map_ns = nullptr, *d_map_nb = nullptr;
    int *d_map_nc = nullptr, *d_map_ng = nullptr;
    int *d_env_map = nullptr, *d_order = nullptr;
    float* d_targets = nullptr;
    float* d_pool = nullptr;
    float *d_drag = nullptr, *d_lam = nullptr;
    int ns_max = 0, nb_max = 0, nc_max = 0, ng_max = 0, n_maps = 0;
    std::vector<int> h_map_ng, h_env_map;  // host copies (gate index checks)
    // sensors
    float4 *d_cam = nullptr, *d_lid = nullptr;
    float *d_cam_tmax = nullptr, *d_lid_tmax = nullptr;
    std::vector<float4> h_dirs[ds::MAX_SENSORS];     // host copies of the body-frame ray tables
    std::vector<float> h_tmax[ds::MAX_SENSORS];
    int img_w[ds::MAX_SENSORS] = {0, 0}, img_h[ds::MAX_SENSORS] = {0, 0};  // ray grid (camera W x H, LiDAR Az x C)
    float4* d_cone[ds::MAX_SENSORS] = {nullptr, nullptr};
    float* d_cone_sin[ds::MAX_SENSORS] = {nullptr, nullptr};
    float4* d_dirp[ds::MAX_SENSORS] = {nullptr, nullptr};  // tile-ordered ray tables of the render kernels
    float* d_tmaxp[ds::MAX_SENSORS] = {nullptr, nullptr};
    int* d_pix[ds::MAX_SENSORS] = {nullptr, nullptr};
    int cull_mode = 1;
    ds::Sensor sen[ds::MAX_SENSORS];
    // state and records
    float* d_state = nullptr;
    int* d_pool_k = nullptr;
    float* d_ckpt = nullptr;
    int* d_ckpt_k = nullptr;
    uint8_t* d_done_tape = nullptr;
    int16_t* d_sdf_tape = nullptr;
    int16_t *d_tape_cam = nullptr, *d_tape_lid = nullptr;
    int* d_gate_k = nullptr;          // [NM] racing: next gate of each agent
    int16_t* d_gate_tape = nullptr;   // [T][NM] racing: gate targeted during each step
    float* d_imu_bias = nullptr;      // [NM][6] IMU bias state
    float *d_poses = nullptr, *d_gposes = nullptr;  // [T][NM][12] rollout poses and their cotangents
    float *d_pose1 = nullptr, *d_gpose1 = nullptr;  // [NM][12] single-step poses and cotangents
    float* d_state2 = nullptr;                       // [NM][D] scratch state of the step adjoint
    int *d_work = nullptr, *d_status = nullptr;
    unsigned long long* d_counters = nullptr;
    size_t bytes = 0;
    bool have_rollout = false;
    const float* rollout_actions = nullptr;
    cudaStream_t last_stream = nullptr;
    // launch shape of the render kernels (forward, adjoint, single-step adjoint)
    int nw = 8, rpt = 4, grid_r = 1, grid_rv = 1, grid_rvs = 1, grid_rvt = 1;
    // ray parts per render item of a rollout and of a single step: enough
    // items per environment for 8 warps (a function of T and M only)
    int parts_roll = 1, parts_one = 1;
    int wait_polls = 0;  // sim_set_wait_limit
    int counting = 1;    // sim_set_counting
    ds::Smem sm_r{}, sm_rv{}, sm_rvs{}, sm_rvt{};
    // kernel launches per kind; while profiling, one CUDA event pair per launch
    bool profiling = false, capturing = false, ev_overflow = false;
    long long launches[SIM_KERNEL_KINDS] = {};
    long long cap_launches[SIM_KERNEL_KINDS] = {};
    struct Ev {
        cudaEvent_t a = nullptr, b = nullptr;
        int kind = 0;
    };
    std::vector<Ev> evs;
    size_t ev_used = 0;
    // advanced by every call that reallocates scene, pool or per-env buffers:
    // a graph captured before such a call refuses to launch
    unsigned generation = 0;
    std::vector<sim_graph*> graphs;
};

// A captured reset + rollout (+ adjoint) of one handle.
struct sim_graph {
    sim_handle* h = nullptr;  // NULL once the handle is destroyed
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned generation = 0;
    const float* actions = nullptr;
    long long launches[SIM_KERNEL_KINDS] = {};
    int kernels = 0;
};

namespace {

const char* kErr[] = {"ok", "invalid argument", "null pointer", "size error", "CUDA error",
                      "not ready", "non-finite state", "device wait timed out", "out of device memory",
                      "unsupported configuration"};

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return SIM_OK;
    if (e == cudaErrorMemoryAllocation) return SIM_ERR_OOM;
    return SIM_ERR_CUDA;
}

#define CK(x)                               \
    do {                                    \
        cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) {            \
            cudaGetLastError();             \
            return cuda_err(e_);            \
        }                                   \
    } while (0)

template <class T>
int dalloc(sim_handle* h, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) return SIM_OK;
    CK(cudaMalloc((void**)p, n * sizeof(T)));
    h->bytes += n * sizeof(T);
    return SIM_OK;
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

int validate(const sim_config* c) {
    if (c->model < SIM_MODEL_POINT_MASS || c->model > SIM_MODEL_SIMPLE) return SIM_ERR_INVALID_ARG;
    if (c->n_env < 1 || c->n_agent < 1 || c->horizon < 1) return SIM_ERR_SIZE;
    if (c->n_agent > 32) return SIM_ERR_SIZE;
    if ((long long)c->n_env * c->n_agent > (1LL << 30)) return SIM_ERR_SIZE;
    if (!finite_pos(c->dt) || !std::isfinite(c->gravity)) return SIM_ERR_INVALID_ARG;
    if (c->model == SIM_MODEL_POINT_MASS || c->model == SIM_MODEL_POINT_MASS_DISCRETE) {
        if (!std::isfinite(c->lam) || !std::isfinite(c->drag) || !std::isfinite(c->act_scale)) return SIM_ERR_INVALID_ARG;
        if (!(c->ema_alpha >= 0.f && c->ema_alpha <= 1.f)) return SIM_ERR_INVALID_ARG;
    } else if (c->model == SIM_MODEL_SIMPLE) {
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(c->rate_scale[i])) return SIM_ERR_INVALID_ARG;
    } else {
        if (!finite_pos(c->mass)) return SIM_ERR_INVALID_ARG;
        for (int i = 0; i < 3; ++i)
            if (!finite_pos(c->inertia[i]) || !std::isfinite(c->k_rate[i]) || !std::isfinite(c->drag_body[i]) ||
                !std::isfinite(c->rate_scale[i]))
                return SIM_ERR_INVALID_ARG;
    }
    if (c->cam_w < 0 || c->cam_h < 0 || c->lid_ch < 0 || c->lid_az < 0) return SIM_ERR_SIZE;
    if (c->cam_w > 0) {
        if (c->cam_h < 1 || (long long)c->cam_w * c->cam_h > (1 << 20)) return SIM_ERR_SIZE;
        if (!(c->cam_hfov > 0.f && c->cam_hfov < 3.1f) || !finite_pos(c->cam_range)) return SIM_ERR_INVALID_ARG;
    }
    if (c->lid_ch > 0) {
        if (c->lid_az < 1 || (long long)c->lid_ch * c->lid_az > (1 << 20)) return SIM_ERR_SIZE;
        if (!finite_pos(c->lid_range) || !(c->lid_elev_lo <= c->lid_elev_hi) || c->lid_elev_lo < -1.5707964f ||
            c->lid_elev_hi > 1.5707964f)
            return SIM_ERR_INVALID_ARG;
    }
    if (c->pool_size < 0 || c->ckpt_every < 0) return SIM_ERR_SIZE;
    if (c->terminate != 0 && c->terminate != 1) return SIM_ERR_INVALID_ARG;
    if (c->tape_hits < -1 || c->tape_hits > 1 || c->cull < -1 || c->cull > 2) return SIM_ERR_INVALID_ARG;
    if (c->warps_per_cta < 0 || c->warps_per_cta > 8) return SIM_ERR_INVALID_ARG;
    {
        // the physics adjoint keeps a segment of (K + 1) states per agent in shared memory
        const long K = c->ckpt_every > 0 ? std::min(c->ckpt_every, c->horizon) : c->horizon;
        if ((K + 1) * (long)c->n_agent * 64 > 200L * 1024) return SIM_ERR_SIZE;
    }
    if (c->rays_per_thread != 0 && !ds::rpt_supported(c->rays_per_thread)) return SIM_ERR_INVALID_ARG;
    if (c->ctas_per_sm < 0) return SIM_ERR_INVALID_ARG;
    if (c->task != SIM_TASK_REACH && c->task != SIM_TASK_RACING) return SIM_ERR_INVALID_ARG;
    for (int i = 0; i < 2; ++i)
        if (!(c->imu_noise[i] >= 0.f) || !(c->imu_walk[i] >= 0.f) || !std::isfinite(c->imu_noise[i]) ||
            !std::isfinite(c->imu_walk[i]))
            return SIM_ERR_INVALID_ARG;
    if (c->cast_mode < 0 || c->cast_mode > 1) return SIM_ERR_INVALID_ARG;
    return SIM_OK;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory of a render CTA: the map block, one cull list per warp, the
// adjoint's hit queue per warp, the TMA barrier.
ds::Smem layout_render(const sim_handle* h, bool lists, bool queues) {
    ds::Smem s{};
    size_t o = 0;
    s.prim = 0;
    const ds::LCap cap{h->ns_max, h->nb_max, h->nc_max, h->ng_max};
    o = align16((size_t)(h->ns_max + 2 * (h->nb_max + h->nc_max + h->ng_max)) * 16);
    s.wlist = (int)o;
    s.wstride = (int)ds::wlist_bytes(cap);
    if (lists) o += (size_t)h->nw * s.wstride;
    s.vq = (int)o;
    if (queues) o += (size_t)h->nw * ds::VQ_BYTES;
    s.mbar = (int)o;
    o += 16;
    s.total = (int)o;
    return s;
}

// Rays per thread: best lane utilisation over the sensors' ray counts (ties
// to more rays per thread, which share each list entry's load).
int pick_rpt(const sim_handle* h) {
    if (h->cfg.rays_per_thread) return h->cfg.rays_per_thread;
    if (h->S == 0) return 1;
    const int cands[] = {8, 6, 5, 4, 3, 2, 1};
    double best = -1.0;
    int pick = 4;
    for (int r : cands) {
        long slots = 0, rays = 0;
        for (int s = 0; s < h->S; ++s) {
            slots += (long)32 * r * ((h->sen[s].R + 32 * r - 1) / (32 * r));
            rays += h->sen[s].R;
        }
        const double util = (double)rays / (double)slots;
        if (util > best + 1e-9) { best = util; pick = r; }
    }
    return pick;
}

int grid_of(sim_handle* h, bool vjp, bool tape, const ds::Smem& sm, int* grid) {
    int occ = 0;
    Args dummy;
    memset(&dummy, 0, sizeof(dummy));
    static int16_t tape_marker;  // selects the taped-adjoint kernel; never dereferenced here
    dummy.sen[0].tape = tape ? &tape_marker : nullptr;
    dummy.nc_max = h->nc_max;  // selects the kernels with cylinders and gates
    dummy.cast_mode = h->cfg.cast_mode;
    dummy.ng_max = h->ng_max;
    CK(ds::render_call(vjp, false, h->rpt, dummy, 0, 32 * h->nw, sm.total, nullptr, &occ));
    if (occ < 1) return SIM_ERR_UNSUPPORTED;
    if (h->cfg.ctas_per_sm) occ = std::min(occ, h->cfg.ctas_per_sm);
    *grid = (int)std::min<long>((long)occ * h->num_sms, h->N);
    return SIM_OK;
}

// Interleaves the bits of x (even positions) and y (odd positions).
uint64_t morton2(uint32_t x, uint32_t y) {
    uint64_t m = 0;
    for (int b = 0; b < 16; ++b) m |= (uint64_t)((x >> b) & 1u) << (2 * b) | (uint64_t)((y >> b) & 1u) << (2 * b + 1);
    return m;
}

// Ray order of the render kernels: a function of the ray grid alone (never
// of rays per thread, culling mode or CTA shape), so every launch shape sums
// the adjoint's ray cotangents in one order and agrees bit for bit.  Grids
// above kMortonMin rays (all of them) take Z (Morton) order, so that each
// chunk of a warp pass covers a compact patch of directions.  Each chunk's cone (body
// frame): axis = normalised mean direction, half-angle = largest angle to
// the axis + 2 mrad.  Tables are uploaded in that order with the output index
// of every slot.  Returns the mean cone half-angle (rad).
constexpr size_t kMortonMin = 0;  // grids above this many rays take Z order

int build_tables(sim_handle* h, int s, double* mean_angle) {
    const int cs = 32 * h->rpt, W = h->img_w[s], H = h->img_h[s];
    std::vector<int> order((size_t)W * H);
    std::iota(order.begin(), order.end(), 0);
    if ((size_t)W * H > kMortonMin)
        std::stable_sort(order.begin(), order.end(), [W](int a, int b) {
            return morton2(a % W, a / W) < morton2(b % W, b / W);
        });
    const std::vector<float4>& d0 = h->h_dirs[s];
    const int R = (int)order.size(), n = (R + cs - 1) / cs;
    std::vector<float4> dirp(R), cone(n);
    std::vector<float> tp(R), sn(n);
    for (int j = 0; j < R; ++j) { dirp[j] = d0[order[j]]; tp[j] = h->h_tmax[s][order[j]]; }
    double sum = 0.0;
    for (int c = 0; c < n; ++c) {
        const int r0 = c * cs, r1 = std::min(R, r0 + cs);
        double ax = 0, ay = 0, az = 0;
        for (int r = r0; r < r1; ++r) { ax += dirp[r].x; ay += dirp[r].y; az += dirp[r].z; }
        const double nn = std::sqrt(ax * ax + ay * ay + az * az);
        double cmin = -1.0;
        if (nn > 1e-9) {
            ax /= nn; ay /= nn; az /= nn;
            cmin = 1.0;
            for (int r = r0; r < r1; ++r)
                cmin = std::min(cmin, (double)dirp[r].x * ax + (double)dirp[r].y * ay + (double)dirp[r].z * az);
        } else {
            ax = 1; ay = 0; az = 0;
        }
        const double th_c = std::min(std::acos(std::max(-1.0, std::min(1.0, cmin))) + 2e-3, M_PI);
        sum += th_c;
        cone[c] = make_float4((float)ax, (float)ay, (float)az, (float)std::cos(th_c));
        sn[c] = (float)std::sin(th_c);
    }
    *mean_angle = sum / n;
    dfree(h->d_cone[s]); dfree(h->d_cone_sin[s]); dfree(h->d_dirp[s]); dfree(h->d_tmaxp[s]); dfree(h->d_pix[s]);
    int rc;
    if ((rc = dalloc(h, &h->d_cone[s], n)) || (rc = dalloc(h, &h->d_cone_sin[s], n)) || (rc = dalloc(h, &h->d_dirp[s], R)) ||
        (rc = dalloc(h, &h->d_tmaxp[s], R)) || (rc = dalloc(h, &h->d_pix[s], R)))
        return rc;
    CK(cudaMemcpy(h->d_cone[s], cone.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_cone_sin[s], sn.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_dirp[s], dirp.data(), R * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_tmaxp[s], tp.data(), R * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_pix[s], order.data(), R * sizeof(int), cudaMemcpyHostToDevice));
    bool identity = true;
    for (int j = 0; j < R && identity; ++j) identity = order[j] == j;
    if (identity) dfree(h->d_pix[s]);  // natural order: no index table
    return SIM_OK;
}

// Half-angle of the cone around all rays of sensor s (pi when their mean
// direction vanishes, as for a full-circle LiDAR).
double sensor_half_angle(const sim_handle* h, int s) {
    const std::vector<float4>& d = h->h_dirs[s];
    double ax = 0, ay = 0, az = 0;
    for (const float4& v : d) { ax += v.x; ay += v.y; az += v.z; }
    const double nn = std::sqrt(ax * ax + ay * ay + az * az);
    if (nn <= 1e-9 * (double)d.size()) return M_PI;
    double cmin = 1.0;
    for (const float4& v : d) cmin = std::min(cmin, (v.x * ax + v.y * ay + v.z * az) / nn);
    return std::min(std::acos(std::max(-1.0, std::min(1.0, cmin))) + 2e-3, M_PI);
}

// Rays per thread and culling mode.  Culling: 0 off, 1 sensor frustum, 2
// frustum + chunk cones.  Chunks of a power-of-two ray count cover whole
// Z-order blocks of the ray grid, so the cones take 4 rays per thread (128
// per chunk) unless the caller fixes it; auto enables them when such a
// chunk's cone is on average under half the sensor's own (ray-weighted over
// the sensors: large camera images and LiDAR scans), else the frustum alone
// with the rays per thread that fill the lanes best.
int configure_launch(sim_handle* h) {
    h->nw = h->cfg.warps_per_cta ? h->cfg.warps_per_cta : 8;
    const int cone_rpt = h->cfg.rays_per_thread ? h->cfg.rays_per_thread : 4;
    int cull = h->cfg.cull;
    if (cull < 0) {
        h->rpt = cone_rpt;
        double num = 0.0, den = 0.0;
        for (int s = 0; s < h->S; ++s) {
            double ang = 0.0;
            int rc = build_tables(h, s, &ang);
            if (rc) return rc;
            num += h->sen[s].R * ang / sensor_half_angle(h, s);
            den += h->sen[s].R;
        }
        cull = den > 0.0 && num < 0.5 * den ? 2 : 1;
    }
    h->rpt = cull == 2 ? cone_rpt : pick_rpt(h);
    for (int s = 0; s < h->S; ++s) {
        double ang = 0.0;
        int rc = build_tables(h, s, &ang);
        if (rc) return rc;
    }
    h->cull_mode = cull;
    h->sm_r = layout_render(h, h->S > 0, false);
    h->sm_rv = layout_render(h, h->S > 0 && !h->tape, h->S > 0);
    h->sm_rvs = layout_render(h, h->S > 0, h->S > 0);
    h->sm_rvt = layout_render(h, false, h->S > 0);
    int maxsm = 0;
    CK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (h->sm_r.total > maxsm || h->sm_rv.total > maxsm || h->sm_rvs.total > maxsm || h->sm_rvt.total > maxsm)
        return SIM_ERR_SIZE;
    int w;
    size_t segb;
    ds::physics_bwd_shape(h->K, h->M, &w, &segb);
    if ((int)segb > maxsm) return SIM_ERR_SIZE;
    int rc;
    if ((rc = grid_of(h, false, false, h->sm_r, &h->grid_r)) ||
        (rc = grid_of(h, true, h->tape, h->sm_rv, &h->grid_rv)) ||
        (rc = grid_of(h, true, false, h->sm_rvs, &h->grid_rvs)) ||
        (rc = grid_of(h, true, true, h->sm_rvt, &h->grid_rvt)))
        return rc;
    return SIM_OK;
}

Args base_args(const sim_handle* h) {
    Args a;
    memset(&a, 0, sizeof(a));
    const sim_config& c = h->cfg;
    a.c.model = c.model; a.c.M = h->M; a.c.D = h->D; a.c.A = h->A;
    a.c.dt = c.dt; a.c.g = c.gravity; a.c.lam = c.lam; a.c.drag = c.drag;
    a.c.act_scale = c.act_scale; a.c.ema_alpha = c.ema_alpha; a.c.mass = c.mass;
    for (int i = 0; i < 3; ++i) {
        a.c.J[i] = c.inertia[i]; a.c.K[i] = c.k_rate[i]; a.c.Dd[i] = c.drag_body[i];
        a.c.rs[i] = c.rate_scale[i]; a.c.blo[i] = c.bound_lo[i]; a.c.bhi[i] = c.bound_hi[i];
    }
    a.c.pos_sq = c.pos_sq; a.c.w_pos = c.w_pos; a.c.w_obs = c.w_obs; a.c.d_safe = c.d_safe;
    a.c.w_act = c.w_act; a.c.w_agent = c.w_agent; a.c.d_agent = c.d_agent;
    a.c.success_radius = c.success_radius; a.c.r_quad = c.r_quad;
    a.c.terminate = c.terminate; a.c.P = h->have_pool ? c.pool_size : 0;
    a.c.task = c.task;
    for (int i = 0; i < 2; ++i) { a.c.imu_noise[i] = c.imu_noise[i]; a.c.imu_walk[i] = c.imu_walk[i]; }
    a.N = h->N; a.M = h->M; a.NM = h->NM; a.T = h->T; a.K = h->K; a.S = h->S;
    a.ns_max = h->ns_max; a.nb_max = h->nb_max; a.cull = h->cull_mode;
    a.cast_mode = h->cfg.cast_mode;
    a.nc_max = h->nc_max; a.ng_max = h->ng_max;
    for (int s = 0; s < ds::MAX_SENSORS; ++s) {
        a.sen[s] = h->sen[s];
        if (s < h->S) {  // the render kernels read the tile-ordered tables
            a.sen[s].dir = h->d_dirp[s];
            a.sen[s].tmax = h->d_tmaxp[s];
            a.sen[s].pix = h->d_pix[s];
            a.sen[s].cone = h->d_cone[s];
            a.sen[s].cone_sin = h->d_cone_sin[s];
        }
    }
    a.prims = h->d_prims; a.map_off = h->d_map_off; a.map_ns = h->d_map_ns; a.map_nb = h->d_map_nb;
    a.map_nc = h->d_map_nc; a.map_ng = h->d_map_ng;
    a.gate_k = h->d_gate_k; a.imu_bias = h->d_imu_bias;
    a.env_map = h->d_env_map; a.order = h->d_order; a.targets = h->d_targets;
    a.pool = h->have_pool ? h->d_pool : nullptr;
    a.drag_env = h->d_drag; a.lam_env = h->d_lam;
    a.state = h->d_state; a.pool_k = h->d_pool_k;
    a.work = h->d_work; a.status = h->d_status;
    a.wait_polls = h->wait_polls;
    a.counters = h->counting ? h->d_counters : nullptr;
    a.parts = h->parts_roll;
    return a;
}

constexpr size_t kMaxEvents = size_t(1) << 16;

// Enqueues one kernel through launch() on st and counts it under `kind`.
// While profiling (and not capturing a graph) the launch is bracketed by a
// CUDA event pair recorded on st, read back by sim_kernel_times.
template <class F>
int launch_kernel(sim_handle* h, int kind, cudaStream_t st, F&& launch) {
    h->last_stream = st;
    size_t slot = SIZE_MAX;
    if (h->profiling && !h->capturing) {
        if (h->ev_used == kMaxEvents) {
            h->ev_overflow = true;
        } else {
            if (h->ev_used == h->evs.size()) {
                sim_handle::Ev e;
                CK(cudaEventCreate(&e.a));
                cudaError_t err = cudaEventCreate(&e.b);
                if (err != cudaSuccess) {
                    cudaEventDestroy(e.a);
                    cudaGetLastError();
                    return cuda_err(err);
                }
                h->evs.push_back(e);
            }
            slot = h->ev_used;
            h->evs[slot].kind = kind;
            CK(cudaEventRecord(h->evs[slot].a, st));
        }
    }
    CK(launch());
    if (slot != SIZE_MAX) {
        CK(cudaEventRecord(h->evs[slot].b, st));
        h->ev_used = slot + 1;
    }
    if (h->capturing) ++h->cap_launches[kind];
    else ++h->launches[kind];
    return SIM_OK;
}

int run_physics(sim_handle* h, const Args& a, cudaStream_t st) {
    return launch_kernel(h, SIM_KERNEL_PHYSICS, st, [&] { return ds::launch_physics(a, st); });
}

int run_physics_bwd(sim_handle* h, const Args& a, cudaStream_t st) {
    return launch_kernel(h, SIM_KERNEL_PHYSICS_BWD, st, [&] { return ds::launch_physics_bwd(a, st); });
}

// Ray parts per (step, agent, sensor) item of the forward render: when an
// environment's T x M x S items are fewer than the CTA's warps, each sensor's
// chunks are split into parts, the warps' worth of parts shared among the
// sensors in proportion to their chunk counts (every part builds its own
// list, so no more parts than warps).
void set_render_parts(const sim_handle* h, Args& a) {
    int nch[ds::MAX_SENSORS] = {0, 0}, tot = 0;
    for (int s = 0; s < h->S; ++s) tot += nch[s] = std::max(1, (h->sen[s].R + 32 * h->rpt - 1) / (32 * h->rpt));
    const int items = a.T * h->M;
    const int want = (h->nw + items - 1) / items;  // parts per (step, agent) over all sensors
    for (int s = 0; s < ds::MAX_SENSORS; ++s) a.rparts[s] = 1;
    if (want <= h->S) return;
    int left = want;
    for (int s = 0; s < h->S; ++s) {
        const int q = s + 1 < h->S ? std::max(1, (int)std::lround((double)want * nch[s] / tot)) : left;
        a.rparts[s] = std::max(1, std::min(q, nch[s]));
        left -= a.rparts[s];
        if (left < h->S - s - 1) left = h->S - s - 1;
    }
}

// which: 0 render, 1 render adjoint (rollout), 2 render adjoint re-casting
// (step), 3 render adjoint gathering caller-supplied hit ids (step)
int run_render(sim_handle* h, int which, Args& a, cudaStream_t st) {
    if (which == 0) set_render_parts(h, a);
    const ds::Smem* sm = which == 0 ? &h->sm_r : (which == 1 ? &h->sm_rv : (which == 2 ? &h->sm_rvs : &h->sm_rvt));
    const int grid = which == 0 ? h->grid_r : (which == 1 ? h->grid_rv : (which == 2 ? h->grid_rvs : h->grid_rvt));
    a.sm = *sm;
    CK(cudaMemsetAsync(h->d_work, 0, sizeof(int), st));
    int occ = 0;
    return launch_kernel(h, which == 0 ? SIM_KERNEL_RENDER : SIM_KERNEL_RENDER_VJP, st, [&] {
        return ds::render_call(which != 0, true, h->rpt, a, grid, 32 * h->nw, sm->total, st, &occ);
    });
}

void build_sensors(sim_handle* h, std::vector<float4>& cam, std::vector<float4>& lid, std::vector<float>& cam_t,
                   std::vector<float>& lid_t) {
    const sim_config& c = h->cfg;
    int s = 0;
    if (c.cam_w > 0) {
        const int W = c.cam_w, H = c.cam_h;
        const double th = std::tan(0.5 * (double)c.cam_hfov), tv = th * H / W;
        double fmin = 1.0;
        cam.resize((size_t)W * H);
        cam_t.resize((size_t)W * H);
        for (int j = 0; j < H; ++j)
            for (int i = 0; i < W; ++i) {
                double u = (2.0 * (i + 0.5) / W - 1.0) * th, v = (2.0 * (j + 0.5) / H - 1.0) * tv;
                double n = std::sqrt(1.0 + u * u + v * v);
                cam[(size_t)j * W + i] = make_float4((float)(1.0 / n), (float)(-u / n), (float)(-v / n), (float)(1.0 / n));
                cam_t[(size_t)j * W + i] = (float)((double)c.cam_range * n);
                fmin = std::min(fmin, 1.0 / n);
            }
        ds::Sensor& S = h->sen[s++];
        S.R = W * H; S.range = c.cam_range; S.kind = 0;
        S.c0 = (float)th; S.c1 = (float)tv;
        S.c2 = (float)(1.0 / std::sqrt(1.0 + th * th)); S.c3 = (float)(1.0 / std::sqrt(1.0 + tv * tv));
        S.maxlen = (float)(c.cam_range / fmin);
    }
    if (c.lid_ch > 0) {
        const int C = c.lid_ch, Az = c.lid_az;
        lid.resize((size_t)C * Az);
        lid_t.assign((size_t)C * Az, c.lid_range);
        for (int ch = 0; ch < C; ++ch) {
            double el = C > 1 ? c.lid_elev_lo + ch * ((double)c.lid_elev_hi - c.lid_elev_lo) / (C - 1)
                              : 0.5 * ((double)c.lid_elev_lo + c.lid_elev_hi);
            for (int k = 0; k < Az; ++k) {
                double az = 2.0 * M_PI * k / Az;
                lid[(size_t)ch * Az + k] = make_float4((float)(std::cos(el) * std::cos(az)),
                                                       (float)(std::cos(el) * std::sin(az)), (float)std::sin(el), 1.f);
            }
        }
        ds::Sensor& S = h->sen[s++];
        S.R = C * Az; S.range = c.lid_range; S.kind = 1;
        S.c0 = c.lid_elev_lo; S.c1 = c.lid_elev_hi;
        S.maxlen = c.lid_range;
    }
    h->S = s;
}

}  // namespace

extern "C" {

const char* sim_version(void) { return "diffsim-b300 0.1 (sm_103a)"; }

const char* sim_strerror(int code) {
    if (code > 0 || code < -9) return "unknown error";
    return kErr[-code];
}

int sim_state_dim(int model) {
    switch (model) {
        case SIM_MODEL_POINT_MASS: case SIM_MODEL_POINT_MASS_DISCRETE: return 12;
        case SIM_MODEL_RIGID: return 13;
        case SIM_MODEL_SIMPLE: return 15;
        default: return -1;
    }
}
int sim_action_dim(int model) {
    switch (model) {
        case SIM_MODEL_POINT_MASS: case SIM_MODEL_POINT_MASS_DISCRETE: return 3;
        case SIM_MODEL_RIGID: case SIM_MODEL_SIMPLE: return 4;
        default: return -1;
    }
}

int sim_destroy(sim_handle* h) {
    if (!h) return SIM_OK;
    cudaDeviceSynchronize();
    for (sim_graph* g : h->graphs) {  // the graph objects stay valid but refuse to launch
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        g->exec = nullptr;
        g->graph = nullptr;
        g->h = nullptr;
    }
    for (auto& e : h->evs) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    dfree(h->d_prims); dfree(h->d_map_off); dfree(h->d_map_ns); dfree(h->d_map_nb);
    dfree(h->d_map_nc); dfree(h->d_map_ng);
    dfree(h->d_gate_k); dfree(h->d_gate_tape); dfree(h->d_imu_bias);
    dfree(h->d_env_map); dfree(h->d_order); dfree(h->d_targets); dfree(h->d_pool);
    dfree(h->d_drag); dfree(h->d_lam); dfree(h->d_cam); dfree(h->d_lid);
    dfree(h->d_cam_tmax); dfree(h->d_lid_tmax);
    for (int s = 0; s < ds::MAX_SENSORS; ++s) {
        dfree(h->d_cone[s]); dfree(h->d_cone_sin[s]); dfree(h->d_dirp[s]); dfree(h->d_tmaxp[s]); dfree(h->d_pix[s]);
    }
    dfree(h->d_state); dfree(h->d_pool_k); dfree(h->d_ckpt); dfree(h->d_ckpt_k);
    dfree(h->d_done_tape); dfree(h->d_sdf_tape); dfree(h->d_tape_cam); dfree(h->d_tape_lid);
    dfree(h->d_poses); dfree(h->d_gposes); dfree(h->d_pose1); dfree(h->d_gpose1); dfree(h->d_state2);
    dfree(h->d_work); dfree(h->d_status); dfree(h->d_counters);
    delete h;
    return SIM_OK;
}

int sim_create(const sim_config* cfg, sim_handle** out) {
    if (!cfg || !out) return SIM_ERR_NULL_PTR;
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    sim_handle* h = new (std::nothrow) sim_handle();
    if (!h) return SIM_ERR_OOM;
    h->cfg = *cfg;
    h->D = sim_state_dim(cfg->model);
    h->A = sim_action_dim(cfg->model);
    h->N = cfg->n_env; h->M = cfg->n_agent; h->NM = h->N * h->M; h->T = cfg->horizon;
    h->K = cfg->ckpt_every > 0 ? std::min(cfg->ckpt_every, h->T) : h->T;
    h->Rc = cfg->cam_w > 0 ? cfg->cam_w * cfg->cam_h : 0;
    h->Rl = cfg->lid_ch > 0 ? cfg->lid_ch * cfg->lid_az : 0;
#define TRY(x)                 \
    do {                       \
        int r_ = (x);          \
        if (r_) {              \
            sim_destroy(h);    \
            return r_;         \
        }                      \
    } while (0)
    TRY(cuda_err(cudaGetDevice(&h->device)));
    TRY(cuda_err(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)));
    std::vector<float4> cam, lid;
    std::vector<float> cam_t, lid_t;
    build_sensors(h, cam, lid, cam_t, lid_t);
    int s = 0;
    if (h->Rc) {
        TRY(dalloc(h, &h->d_cam, cam.size()));
        TRY(dalloc(h, &h->d_cam_tmax, cam_t.size()));
        TRY(cuda_err(cudaMemcpy(h->d_cam, cam.data(), cam.size() * sizeof(float4), cudaMemcpyHostToDevice)));
        TRY(cuda_err(cudaMemcpy(h->d_cam_tmax, cam_t.data(), cam_t.size() * sizeof(float), cudaMemcpyHostToDevice)));
        h->sen[s].dir = h->d_cam;
        h->h_dirs[s] = cam;
        h->h_tmax[s] = cam_t;
        h->img_w[s] = cfg->cam_w;
        h->img_h[s] = cfg->cam_h;
        h->sen[s++].tmax = h->d_cam_tmax;
    }
    if (h->Rl) {
        TRY(dalloc(h, &h->d_lid, lid.size()));
        TRY(dalloc(h, &h->d_lid_tmax, lid_t.size()));
        TRY(cuda_err(cudaMemcpy(h->d_lid, lid.data(), lid.size() * sizeof(float4), cudaMemcpyHostToDevice)));
        TRY(cuda_err(cudaMemcpy(h->d_lid_tmax, lid_t.data(), lid_t.size() * sizeof(float), cudaMemcpyHostToDevice)));
        h->sen[s].dir = h->d_lid;
        h->h_dirs[s] = lid;
        h->h_tmax[s] = lid_t;
        h->img_w[s] = cfg->lid_az;
        h->img_h[s] = cfg->lid_ch;
        h->sen[s++].tmax = h->d_lid_tmax;
    }
    // ray-adjoint items per environment: enough for every lane group of a
    // CTA of 8 warps (VQ_PER_WARP items per warp) when the horizon and the
    // agents give fewer (step, agent) items; fixed, so that every launch
    // shape splits the rays alike and gives the same sums
    const int want = ds::VQ_PER_WARP * 8;
    h->parts_roll = std::min(want, std::max(1, (want + h->T * h->M - 1) / (h->T * h->M)));
    h->parts_one = std::min(want, std::max(1, (want + h->M - 1) / h->M));
    const size_t tape_bytes = (size_t)h->T * h->NM * (h->Rc + h->Rl) * 2;
    h->tape = cfg->tape_hits == 1 || (cfg->tape_hits == -1 && tape_bytes <= (size_t(8) << 30));
    if (h->S == 0) h->tape = false;
    const int nseg = (h->T + h->K - 1) / h->K;
    TRY(dalloc(h, &h->d_state, (size_t)h->NM * h->D));
    TRY(dalloc(h, &h->d_pool_k, (size_t)h->N));
    TRY(dalloc(h, &h->d_ckpt, (size_t)nseg * h->NM * h->D));
    TRY(dalloc(h, &h->d_ckpt_k, (size_t)nseg * h->N));
    TRY(dalloc(h, &h->d_done_tape, (size_t)h->T * h->NM));
    TRY(dalloc(h, &h->d_sdf_tape, (size_t)h->T * h->NM));
    TRY(dalloc(h, &h->d_gate_k, (size_t)h->NM));
    TRY(dalloc(h, &h->d_imu_bias, (size_t)h->NM * 6));
    if (cfg->task == SIM_TASK_RACING) TRY(dalloc(h, &h->d_gate_tape, (size_t)h->T * h->NM));
    TRY(cuda_err(cudaMemset(h->d_gate_k, 0, sizeof(int) * h->NM)));
    TRY(cuda_err(cudaMemset(h->d_imu_bias, 0, sizeof(float) * 6 * h->NM)));
    if (h->tape) {
        if (h->Rc) TRY(dalloc(h, &h->d_tape_cam, (size_t)h->T * h->NM * h->Rc));
        if (h->Rl) TRY(dalloc(h, &h->d_tape_lid, (size_t)h->T * h->NM * h->Rl));
    }
    TRY(dalloc(h, &h->d_poses, (size_t)h->T * h->NM * 12));
    TRY(dalloc(h, &h->d_gposes, (size_t)h->T * h->NM * h->parts_roll * 12));
    TRY(dalloc(h, &h->d_pose1, (size_t)h->NM * 12));
    TRY(dalloc(h, &h->d_gpose1, (size_t)h->NM * h->parts_one * 12));
    TRY(dalloc(h, &h->d_state2, (size_t)h->NM * h->D));
    TRY(dalloc(h, &h->d_work, 1));
    TRY(dalloc(h, &h->d_status, 1));
    TRY(dalloc(h, &h->d_counters, 4));
    TRY(cuda_err(cudaMemset(h->d_status, 0, sizeof(int))));
    TRY(cuda_err(cudaMemset(h->d_counters, 0, 4 * sizeof(unsigned long long))));
    TRY(cuda_err(cudaMemset(h->d_pool_k, 0, sizeof(int) * h->N)));
    TRY(cuda_err(cudaMemset(h->d_state, 0, sizeof(float) * (size_t)h->NM * h->D)));
#undef TRY
    *out = h;
    return SIM_OK;
}

int sim_workspace_bytes(const sim_handle* h, size_t* bytes) {
    if (!h || !bytes) return SIM_ERR_NULL_PTR;
    *bytes = h->bytes;
    return SIM_OK;
}

int sim_set_scene(sim_handle* h, const float* spheres, const int32_t* sph_off, const float* boxes,
                  const int32_t* box_off, int32_t n_maps, const int32_t* env_map, const float* targets) {
    sim_scene sc{};
    sc.n_maps = n_maps;
    sc.spheres = spheres; sc.sph_off = sph_off;
    sc.boxes = boxes; sc.box_off = box_off;
    sc.env_map = env_map; sc.targets = targets;
    return sim_set_scene_ex(h, &sc);
}

namespace {
// Counts of one kind per map from its CSR offsets (all zero when absent);
// false when the offsets are inconsistent.
bool kind_counts(const int32_t* off, int n_maps, std::vector<int>& cnt) {
    cnt.assign(n_maps, 0);
    if (!off) return true;
    if (off[0] != 0) return false;
    for (int m = 0; m < n_maps; ++m) {
        cnt[m] = off[m + 1] - off[m];
        if (cnt[m] < 0) return false;
    }
    return true;
}

bool all_finite(const float* x, long n) {
    for (long k = 0; k < n; ++k)
        if (!std::isfinite(x[k])) return false;
    return true;
}
}  // namespace

int sim_set_scene_ex(sim_handle* h, const sim_scene* sc) {
    if (!h || !sc) return SIM_ERR_NULL_PTR;
    const int n_maps = sc->n_maps;
    if (!sc->sph_off || !sc->box_off || !sc->env_map || !sc->targets) return SIM_ERR_NULL_PTR;
    if ((sc->cylinders != nullptr) != (sc->cyl_off != nullptr) || (sc->gates != nullptr) != (sc->gate_off != nullptr))
        return SIM_ERR_NULL_PTR;
    if (n_maps < 1) return SIM_ERR_SIZE;
    std::vector<int> vns, vnb, vnc, vng;
    if (!kind_counts(sc->sph_off, n_maps, vns) || !kind_counts(sc->box_off, n_maps, vnb) ||
        !kind_counts(sc->cyl_off, n_maps, vnc) || !kind_counts(sc->gate_off, n_maps, vng))
        return SIM_ERR_SIZE;
    int ns_max = 0, nb_max = 0, nc_max = 0, ng_max = 0;
    for (int m = 0; m < n_maps; ++m) {
        if ((long)vns[m] + vnb[m] + vnc[m] + vng[m] > 32767) return SIM_ERR_SIZE;
        if (vnc[m] > 0xffff || vng[m] > 0x7fff) return SIM_ERR_SIZE;
        if (h->cfg.task == SIM_TASK_RACING && vng[m] < 1) return SIM_ERR_SIZE;
        ns_max = std::max(ns_max, vns[m]);
        nb_max = std::max(nb_max, vnb[m]);
        nc_max = std::max(nc_max, vnc[m]);
        ng_max = std::max(ng_max, vng[m]);
    }
    const long Ks = sc->sph_off[n_maps], Kb = sc->box_off[n_maps];
    const long Kc = sc->cyl_off ? sc->cyl_off[n_maps] : 0, Kg = sc->gate_off ? sc->gate_off[n_maps] : 0;
    if ((Ks > 0 && !sc->spheres) || (Kb > 0 && !sc->boxes)) return SIM_ERR_NULL_PTR;
    if (!all_finite(sc->spheres, 4 * Ks) || !all_finite(sc->boxes, 6 * Kb) || !all_finite(sc->cylinders, 5 * Kc) ||
        !all_finite(sc->gates, 7 * Kg))
        return SIM_ERR_INVALID_ARG;
    for (long k = 0; k < Ks; ++k)
        if (sc->spheres[4 * k + 3] < 0.f) return SIM_ERR_INVALID_ARG;
    for (long k = 0; k < Kb; ++k)
        for (int j = 0; j < 3; ++j)
            if (sc->boxes[6 * k + 3 + j] < sc->boxes[6 * k + j]) return SIM_ERR_INVALID_ARG;
    for (long k = 0; k < Kc; ++k)
        if (sc->cylinders[5 * k + 2] < 0.f || sc->cylinders[5 * k + 4] < sc->cylinders[5 * k + 3])
            return SIM_ERR_INVALID_ARG;
    for (long k = 0; k < Kg; ++k)
        if (!(sc->gates[7 * k + 4] > 0.f && sc->gates[7 * k + 5] > 0.f && sc->gates[7 * k + 6] > 0.f))
            return SIM_ERR_INVALID_ARG;
    for (int e = 0; e < h->N; ++e)
        if (sc->env_map[e] < 0 || sc->env_map[e] >= n_maps) return SIM_ERR_SIZE;
    if (!all_finite(sc->targets, 3L * h->NM)) return SIM_ERR_INVALID_ARG;
    // map blocks: spheres (c, r); boxes (min, 0), (max, 0); cylinders
    // (cx, cy, r, 0), (zmin, zmax, 0, 0); gates (c, w), (cos yaw, sin yaw, b, hd)
    std::vector<float4> blk;
    std::vector<int> off(n_maps);
    blk.reserve((size_t)Ks + 2 * (Kb + Kc + Kg));
    for (int m = 0; m < n_maps; ++m) {
        off[m] = (int)blk.size();
        for (int k = sc->sph_off[m]; k < sc->sph_off[m + 1]; ++k) {
            const float* q = sc->spheres + 4 * k;
            blk.push_back(make_float4(q[0], q[1], q[2], q[3]));
        }
        for (int k = sc->box_off[m]; k < sc->box_off[m + 1]; ++k) {
            const float* q = sc->boxes + 6 * k;
            blk.push_back(make_float4(q[0], q[1], q[2], 0.f));
            blk.push_back(make_float4(q[3], q[4], q[5], 0.f));
        }
        for (int k = sc->cyl_off ? sc->cyl_off[m] : 0; sc->cyl_off && k < sc->cyl_off[m + 1]; ++k) {
            const float* q = sc->cylinders + 5 * k;
            blk.push_back(make_float4(q[0], q[1], q[2], 0.f));
            blk.push_back(make_float4(q[3], q[4], 0.f, 0.f));
        }
        for (int k = sc->gate_off ? sc->gate_off[m] : 0; sc->gate_off && k < sc->gate_off[m + 1]; ++k) {
            const float* q = sc->gates + 7 * k;
            blk.push_back(make_float4(q[0], q[1], q[2], q[4]));
            blk.push_back(make_float4((float)std::cos((double)q[3]), (float)std::sin((double)q[3]), q[5], q[6]));
        }
    }
    if (blk.size() >= (size_t)INT32_MAX) return SIM_ERR_SIZE;
    // environments in descending work order (load balance of the ticket queue)
    std::vector<int> order(h->N);
    std::iota(order.begin(), order.end(), 0);
    auto work = [&](int e) {
        const int m = sc->env_map[e];
        return vns[m] + vnb[m] + 2 * (vnc[m] + vng[m]);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
    ++h->generation;
    dfree(h->d_prims); dfree(h->d_map_off); dfree(h->d_map_ns); dfree(h->d_map_nb);
    dfree(h->d_map_nc); dfree(h->d_map_ng);
    dfree(h->d_env_map); dfree(h->d_order); dfree(h->d_targets);
    int rc;
    if ((rc = dalloc(h, &h->d_prims, std::max<size_t>(blk.size(), 1)))) return rc;
    if ((rc = dalloc(h, &h->d_map_off, n_maps)) || (rc = dalloc(h, &h->d_map_ns, n_maps)) ||
        (rc = dalloc(h, &h->d_map_nb, n_maps)) || (rc = dalloc(h, &h->d_env_map, h->N)) ||
        (rc = dalloc(h, &h->d_order, h->N)) || (rc = dalloc(h, &h->d_targets, 3 * (size_t)h->NM)))
        return rc;
    const bool extra = nc_max > 0 || ng_max > 0;
    if (extra && ((rc = dalloc(h, &h->d_map_nc, n_maps)) || (rc = dalloc(h, &h->d_map_ng, n_maps)))) return rc;
    if (!blk.empty()) CK(cudaMemcpy(h->d_prims, blk.data(), blk.size() * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_map_off, off.data(), n_maps * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_map_ns, vns.data(), n_maps * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_map_nb, vnb.data(), n_maps * sizeof(int), cudaMemcpyHostToDevice));
    if (extra) {
        CK(cudaMemcpy(h->d_map_nc, vnc.data(), n_maps * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->d_map_ng, vng.data(), n_maps * sizeof(int), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(h->d_env_map, sc->env_map, h->N * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_order, order.data(), h->N * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_targets, sc->targets, 3 * (size_t)h->NM * sizeof(float), cudaMemcpyHostToDevice));
    h->ns_max = ns_max;
    h->nb_max = nb_max;
    h->nc_max = nc_max;
    h->ng_max = ng_max;
    h->n_maps = n_maps;
    h->h_map_ng = vng;
    h->h_env_map.assign(sc->env_map, sc->env_map + h->N);
    rc = configure_launch(h);
    if (rc) return rc;
    // gate indices start at the first gate
    CK(cudaMemset(h->d_gate_k, 0, sizeof(int) * h->NM));
    h->have_scene = true;
    h->have_rollout = false;
    return SIM_OK;
}

int sim_set_pool(sim_handle* h, const float* pool) {
    if (!h || !pool) return SIM_ERR_NULL_PTR;
    const size_t n = (size_t)h->cfg.pool_size * h->NM * h->D;
    if (n == 0) return SIM_ERR_SIZE;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(pool[k])) return SIM_ERR_INVALID_ARG;
    ++h->generation;
    dfree(h->d_pool);
    int rc = dalloc(h, &h->d_pool, n);
    if (rc) return rc;
    CK(cudaMemcpy(h->d_pool, pool, n * sizeof(float), cudaMemcpyHostToDevice));
    h->have_pool = true;
    return SIM_OK;
}

int sim_set_env_params(sim_handle* h, const float* drag, const float* lam) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (h->cfg.model != SIM_MODEL_POINT_MASS && (drag || lam)) return SIM_ERR_UNSUPPORTED;
    ++h->generation;
    dfree(h->d_drag);
    dfree(h->d_lam);
    int rc;
    if (drag) {
        for (int e = 0; e < h->N; ++e)
            if (!std::isfinite(drag[e])) return SIM_ERR_INVALID_ARG;
        if ((rc = dalloc(h, &h->d_drag, h->N))) return rc;
        CK(cudaMemcpy(h->d_drag, drag, h->N * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (lam) {
        for (int e = 0; e < h->N; ++e)
            if (!std::isfinite(lam[e])) return SIM_ERR_INVALID_ARG;
        if ((rc = dalloc(h, &h->d_lam, h->N))) return rc;
        CK(cudaMemcpy(h->d_lam, lam, h->N * sizeof(float), cudaMemcpyHostToDevice));
    }
    return SIM_OK;
}

int sim_reset(sim_handle* h, const float* state0, sim_stream_t stream) {
    if (!h) return SIM_ERR_NULL_PTR;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->NM * h->D * sizeof(float);
    if (state0) CK(cudaMemcpyAsync(h->d_state, state0, n, cudaMemcpyDeviceToDevice, st));
    else if (h->have_pool) CK(cudaMemcpyAsync(h->d_state, h->d_pool, n, cudaMemcpyDeviceToDevice, st));
    else return SIM_ERR_NOT_READY;
    CK(cudaMemsetAsync(h->d_pool_k, 0, sizeof(int) * h->N, st));
    CK(cudaMemsetAsync(h->d_gate_k, 0, sizeof(int) * h->NM, st));
    CK(cudaMemsetAsync(h->d_imu_bias, 0, sizeof(float) * 6 * h->NM, st));
    h->have_rollout = false;
    h->last_stream = st;
    return SIM_OK;
}

int sim_get_gate_index(const sim_handle* h, int32_t* gate_k, sim_stream_t stream) {
    if (!h || !gate_k) return SIM_ERR_NULL_PTR;
    CK(cudaMemcpyAsync(gate_k, h->d_gate_k, sizeof(int) * h->NM, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SIM_OK;
}

int sim_set_gate_index(sim_handle* h, const int32_t* gate_k, sim_stream_t stream) {
    if (!h || !gate_k) return SIM_ERR_NULL_PTR;
    if (h->cfg.task != SIM_TASK_RACING) return SIM_ERR_UNSUPPORTED;
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    // indices must name a gate of the agent's map: checked on the host
    std::vector<int> k(h->NM);
    CK(cudaMemcpyAsync(k.data(), gate_k, sizeof(int) * h->NM, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; i < h->NM; ++i)
        if (k[i] < 0 || k[i] >= h->h_map_ng[h->h_env_map[i / h->M]]) return SIM_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(h->d_gate_k, gate_k, sizeof(int) * h->NM, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    h->have_rollout = false;
    return SIM_OK;
}

int sim_get_state(const sim_handle* h, float* dst, sim_stream_t stream) {
    if (!h || !dst) return SIM_ERR_NULL_PTR;
    CK(cudaMemcpyAsync(dst, h->d_state, (size_t)h->NM * h->D * sizeof(float), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return SIM_OK;
}

int sim_set_state(sim_handle* h, const float* src, sim_stream_t stream) {
    if (!h || !src) return SIM_ERR_NULL_PTR;
    CK(cudaMemcpyAsync(h->d_state, src, (size_t)h->NM * h->D * sizeof(float), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    h->have_rollout = false;
    return SIM_OK;
}

int sim_get_reset_counters(const sim_handle* h, int32_t* dst, sim_stream_t stream) {
    if (!h || !dst) return SIM_ERR_NULL_PTR;
    CK(cudaMemcpyAsync(dst, h->d_pool_k, (size_t)h->N * sizeof(int), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    return SIM_OK;
}

int sim_set_reset_counters(sim_handle* h, const int32_t* src, sim_stream_t stream) {
    if (!h || !src) return SIM_ERR_NULL_PTR;
    CK(cudaMemcpyAsync(h->d_pool_k, src, (size_t)h->N * sizeof(int), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
    h->have_rollout = false;
    return SIM_OK;
}

int sim_render_taped(sim_handle* h, float* depth, float* lidar, int16_t* hits_cam, int16_t* hits_lidar,
                     sim_stream_t stream) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.render_only = 1;
    a.T = 1;
    a.parts = h->parts_one;
    a.poses = h->d_pose1;
    int rc = run_physics(h, a, st);
    if (rc || h->S == 0) return rc;
    int s = 0;
    if (h->Rc) { a.sen[s].out = depth; a.sen[s].tape = hits_cam; ++s; }
    if (h->Rl) { a.sen[s].out = lidar; a.sen[s].tape = hits_lidar; ++s; }
    return run_render(h, 0, a, st);
}

int sim_render(sim_handle* h, float* depth, float* lidar, sim_stream_t stream) {
    return sim_render_taped(h, depth, lidar, nullptr, nullptr, stream);
}

int sim_render_hits(sim_handle* h, const int16_t* hits_cam, const int16_t* hits_lidar, float* depth, float* lidar,
                    sim_stream_t stream) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    if ((h->Rc && depth && !hits_cam) || (h->Rl && lidar && !hits_lidar)) return SIM_ERR_NULL_PTR;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.render_only = 1;
    a.T = 1;
    a.poses = h->d_pose1;
    int rc = run_physics(h, a, st);
    if (rc || h->S == 0) return rc;
    int s = 0;
    if (h->Rc) { a.sen[s].out = depth; a.sen[s].tape = const_cast<int16_t*>(hits_cam); ++s; }
    if (h->Rl) { a.sen[s].out = lidar; a.sen[s].tape = const_cast<int16_t*>(hits_lidar); ++s; }
    const int grid = std::max(1, std::min(h->NM, h->num_sms * 8));
    return launch_kernel(h, SIM_KERNEL_RENDER, st, [&] { return ds::launch_render_hits(a, grid, st); });
}

int sim_step_ex(sim_handle* h, const sim_rollout_io* io, sim_stream_t stream) {
    if (!h || !io || !io->actions) return SIM_ERR_NULL_PTR;
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    if (h->cfg.terminate && !h->have_pool) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.T = 1;
    a.parts = h->parts_one;
    a.K = 1;
    a.actions = io->actions;
    a.r_ctrl = io->r_ctrl; a.r_goal = io->r_goal; a.done = io->done;
    a.imu = io->imu; a.imu_noise = io->imu_noise;
    a.poses = h->d_pose1;
    int rc = run_physics(h, a, st);
    if (rc || h->S == 0) return rc;
    int s = 0;
    if (h->Rc) { a.sen[s].out = io->depth; a.sen[s].tape = io->hits_cam; ++s; }
    if (h->Rl) { a.sen[s].out = io->lidar; a.sen[s].tape = io->hits_lidar; ++s; }
    return run_render(h, 0, a, st);
}

int sim_step(sim_handle* h, const float* actions, float* depth, float* lidar, float* r_ctrl, int8_t* r_goal,
             uint8_t* done, sim_stream_t stream) {
    sim_rollout_io io{};
    io.actions = actions;
    io.r_ctrl = r_ctrl; io.r_goal = r_goal; io.done = done;
    io.depth = depth; io.lidar = lidar;
    return sim_step_ex(h, &io, stream);
}

int sim_rollout_ex(sim_handle* h, const sim_rollout_io* io, sim_stream_t stream) {
    if (!h || !io || !io->actions) return SIM_ERR_NULL_PTR;
    if (io->hits_cam || io->hits_lidar) return SIM_ERR_INVALID_ARG;  // the rollout tapes its hits itself
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    if (h->cfg.terminate && !h->have_pool) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.actions = io->actions;
    a.r_ctrl = io->r_ctrl; a.r_goal = io->r_goal; a.done = io->done;
    a.imu = io->imu; a.imu_noise = io->imu_noise;
    a.done_tape = h->d_done_tape;
    a.sdf_tape = h->d_sdf_tape;
    a.gate_tape = h->d_gate_tape;
    a.ckpt = h->d_ckpt;
    a.ckpt_k = h->d_ckpt_k;
    a.poses = h->d_poses;
    int rc = run_physics(h, a, st);
    if (rc) return rc;
    if (h->S > 0) {
        int s = 0;
        if (h->Rc) { a.sen[s].out = io->depth; a.sen[s].tape = h->d_tape_cam; ++s; }
        if (h->Rl) { a.sen[s].out = io->lidar; a.sen[s].tape = h->d_tape_lid; ++s; }
        rc = run_render(h, 0, a, st);
        if (rc) return rc;
    }
    h->have_rollout = true;
    h->rollout_actions = io->actions;
    return SIM_OK;
}

int sim_rollout(sim_handle* h, const float* actions, float* r_ctrl, int8_t* r_goal, uint8_t* done, float* depth,
                float* lidar, sim_stream_t stream) {
    sim_rollout_io io{};
    io.actions = actions;
    io.r_ctrl = r_ctrl; io.r_goal = r_goal; io.done = done;
    io.depth = depth; io.lidar = lidar;
    return sim_rollout_ex(h, &io, stream);
}

int sim_backward_ex(sim_handle* h, const sim_grad_io* io, sim_stream_t stream) {
    if (!h || !io || !io->g_r || !io->g_a) return SIM_ERR_NULL_PTR;
    if (!h->have_rollout) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.actions = h->rollout_actions;
    a.done_rd = h->d_done_tape;
    a.sdf_tape = h->d_sdf_tape;
    a.gate_tape = h->d_gate_tape;
    a.ckpt = h->d_ckpt;
    a.ckpt_k = h->d_ckpt_k;
    a.poses = h->d_poses;
    a.g_r = io->g_r; a.g_sT = io->g_sT; a.g_a = io->g_a; a.g_s0 = io->g_s0;
    a.g_imu = io->g_imu;
    int s = 0;
    if (h->Rc) { a.sen[s].gout = io->g_depth; a.sen[s].tape = h->d_tape_cam; ++s; }
    if (h->Rl) { a.sen[s].gout = io->g_lidar; a.sen[s].tape = h->d_tape_lid; ++s; }
    if (h->S > 0 && (io->g_depth || io->g_lidar)) {
        a.gposes = h->d_gposes;
        int rc = run_render(h, 1, a, st);
        if (rc) return rc;
    }
    return run_physics_bwd(h, a, st);
}

int sim_backward(sim_handle* h, const float* g_r, const float* g_depth, const float* g_lidar, const float* g_sT,
                 float* g_a, float* g_s0, sim_stream_t stream) {
    sim_grad_io io{};
    io.g_r = g_r; io.g_depth = g_depth; io.g_lidar = g_lidar; io.g_sT = g_sT;
    io.g_a = g_a; io.g_s0 = g_s0;
    return sim_backward_ex(h, &io, stream);
}

int sim_step_backward_taped(sim_handle* h, const float* s_t, const float* a_t, const uint8_t* done_t,
                            const float* g_s_next, const float* g_r, const float* g_depth, const float* g_lidar,
                            const int16_t* hits_cam, const int16_t* hits_lidar, float* g_a, float* g_s,
                            sim_stream_t stream) {
    if (!h || !s_t || !a_t || !done_t || !g_r || !g_a) return SIM_ERR_NULL_PTR;
    if (!h->have_scene) return SIM_ERR_NOT_READY;
    if (h->cfg.task != SIM_TASK_REACH) return SIM_ERR_UNSUPPORTED;
    const bool taped = hits_cam || hits_lidar;
    if (taped && ((h->Rc && g_depth && !hits_cam) || (h->Rl && g_lidar && !hits_lidar))) return SIM_ERR_NULL_PTR;
    cudaStream_t st = (cudaStream_t)stream;
    Args a = base_args(h);
    a.T = 1;
    a.parts = h->parts_one;
    a.K = 1;
    a.actions = a_t;
    if (h->S > 0 && (g_depth || g_lidar)) {
        // pose after the step, from a scratch copy of s_t (the current state is untouched)
        CK(cudaMemcpyAsync(h->d_state2, s_t, (size_t)h->NM * h->D * sizeof(float), cudaMemcpyDeviceToDevice, st));
        Args f = a;
        f.state = h->d_state2;
        f.pool_k = nullptr;
        f.poses = h->d_pose1;
        int rc = run_physics(h, f, st);
        if (rc) return rc;
        a.poses = h->d_pose1;
        a.gposes = h->d_gpose1;
        a.done_rd = done_t;
        int s = 0;
        if (h->Rc) { a.sen[s].gout = g_depth; a.sen[s].tape = const_cast<int16_t*>(hits_cam); ++s; }
        if (h->Rl) { a.sen[s].gout = g_lidar; a.sen[s].tape = const_cast<int16_t*>(hits_lidar); ++s; }
        rc = run_render(h, taped ? 3 : 2, a, st);
        if (rc) return rc;
    }
    a.done_rd = done_t;
    a.sdf_tape = nullptr;
    a.ckpt = const_cast<float*>(s_t);
    a.ckpt_k = nullptr;
    a.g_r = g_r; a.g_sT = g_s_next; a.g_a = g_a; a.g_s0 = g_s;
    return run_physics_bwd(h, a, st);
}

int sim_step_backward(sim_handle* h, const float* s_t, const float* a_t, const uint8_t* done_t,
                      const float* g_s_next, const float* g_r, const float* g_depth, const float* g_lidar,
                      float* g_a, float* g_s, sim_stream_t stream) {
    return sim_step_backward_taped(h, s_t, a_t, done_t, g_s_next, g_r, g_depth, g_lidar, nullptr, nullptr, g_a,
                                   g_s, stream);
}

int sim_last_status(sim_handle* h, int32_t* status, int32_t* per_env) {
    if (!h || !status) return SIM_ERR_NULL_PTR;
    if (per_env) return SIM_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->last_stream));
    int v = 0;
    CK(cudaMemcpy(&v, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(h->d_status, 0, sizeof(int)));
    *status = v;
    if (v & SIM_STATUS_TIMEOUT) return SIM_ERR_TIMEOUT;
    if (v & SIM_STATUS_NAN) return SIM_ERR_NAN;
    return SIM_OK;
}

int sim_set_wait_limit(sim_handle* h, int32_t polls) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (polls < 0) return SIM_ERR_INVALID_ARG;
    h->wait_polls = polls;
    return SIM_OK;
}

int sim_set_counting(sim_handle* h, int32_t on) {
    if (!h) return SIM_ERR_NULL_PTR;
    h->counting = on != 0;
    return SIM_OK;
}

int sim_counters(sim_handle* h, uint64_t* out, int32_t reset) {
    if (!h || !out) return SIM_ERR_NULL_PTR;
    CK(cudaStreamSynchronize(h->last_stream));
    unsigned long long v[4];
    CK(cudaMemcpy(v, h->d_counters, sizeof(v), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) out[i] = v[i];
    if (reset) CK(cudaMemset(h->d_counters, 0, sizeof(v)));
    return SIM_OK;
}

int sim_launch_info(const sim_handle* h, int32_t* warps_per_cta, int32_t* rays_per_thread, int32_t* grid,
                    int32_t* smem_bytes) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (warps_per_cta) *warps_per_cta = h->nw;
    if (rays_per_thread) *rays_per_thread = h->rpt;
    if (grid) *grid = h->grid_r;
    if (smem_bytes) *smem_bytes = (int32_t)h->sm_r.total;
    return SIM_OK;
}


int sim_profile(sim_handle* h, int32_t on) {
    if (!h) return SIM_ERR_NULL_PTR;
    h->profiling = on != 0;
    return SIM_OK;
}

int sim_kernel_times(sim_handle* h, double* ms, int64_t* launches, int32_t reset) {
    if (!h) return SIM_ERR_NULL_PTR;
    if (ms) {
        for (int k = 0; k < SIM_KERNEL_KINDS; ++k) ms[k] = 0.0;
        for (size_t i = 0; i < h->ev_used; ++i) {
            const sim_handle::Ev& e = h->evs[i];
            CK(cudaEventSynchronize(e.b));
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, e.a, e.b));
            ms[e.kind] += t;
        }
    }
    if (launches)
        for (int k = 0; k < SIM_KERNEL_KINDS; ++k) launches[k] = h->launches[k];
    const bool overflow = h->ev_overflow;
    if (reset) {
        h->ev_used = 0;
        h->ev_overflow = false;
        for (int k = 0; k < SIM_KERNEL_KINDS; ++k) h->launches[k] = 0;
    }
    return overflow ? SIM_ERR_SIZE : SIM_OK;
}

int sim_graph_create(sim_handle* h, const sim_graph_io* io, sim_graph** out) {
    if (!h || !io || !out) return SIM_ERR_NULL_PTR;
    *out = nullptr;
    if (!io->actions || (io->g_r && !io->g_a)) return SIM_ERR_NULL_PTR;
    if (!h->have_scene || (!io->state0 && !h->have_pool)) return SIM_ERR_NOT_READY;
    if (h->cfg.terminate && !h->have_pool) return SIM_ERR_NOT_READY;
    sim_graph* g = new (std::nothrow) sim_graph();
    if (!g) return SIM_ERR_OOM;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return cuda_err(e);
    }
    const bool had_rollout = h->have_rollout;
    const float* had_actions = h->rollout_actions;
    cudaStream_t had_stream = h->last_stream;
    h->capturing = true;
    for (int k = 0; k < SIM_KERNEL_KINDS; ++k) h->cap_launches[k] = 0;
    int rc = cuda_err(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    if (!rc) {
        rc = sim_reset(h, io->state0, cs);
        if (!rc) rc = sim_rollout(h, io->actions, io->r_ctrl, io->r_goal, io->done, io->depth, io->lidar, cs);
        if (!rc && io->g_r) rc = sim_backward(h, io->g_r, io->g_depth, io->g_lidar, io->g_sT, io->g_a, io->g_s0, cs);
        e = cudaStreamEndCapture(cs, &g->graph);  // ends the capture whatever happened inside
        if (!rc && e != cudaSuccess) rc = cuda_err(e);
    }
    h->capturing = false;
    h->have_rollout = had_rollout;
    h->rollout_actions = had_actions;
    h->last_stream = had_stream;
    if (!rc) rc = cuda_err(cudaGraphInstantiate(&g->exec, g->graph, 0));
    if (!rc) {
        size_t n = 0;
        rc = cuda_err(cudaGraphGetNodes(g->graph, nullptr, &n));
        std::vector<cudaGraphNode_t> nodes(n);
        if (!rc && n) rc = cuda_err(cudaGraphGetNodes(g->graph, nodes.data(), &n));
        for (size_t i = 0; !rc && i < n; ++i) {
            cudaGraphNodeType t;
            rc = cuda_err(cudaGraphNodeGetType(nodes[i], &t));
            if (!rc && t == cudaGraphNodeTypeKernel) ++g->kernels;
        }
    }
    cudaStreamDestroy(cs);
    if (rc) {
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc;
    }
    g->h = h;
    g->generation = h->generation;
    g->actions = io->actions;
    for (int k = 0; k < SIM_KERNEL_KINDS; ++k) g->launches[k] = h->cap_launches[k];
    h->graphs.push_back(g);
    *out = g;
    return SIM_OK;
}

int sim_graph_launch(sim_graph* g, sim_stream_t stream) {
    if (!g) return SIM_ERR_NULL_PTR;
    sim_handle* h = g->h;
    if (!h || g->generation != h->generation) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaGraphLaunch(g->exec, st));
    h->last_stream = st;
    h->have_rollout = true;
    h->rollout_actions = g->actions;
    for (int k = 0; k < SIM_KERNEL_KINDS; ++k) h->launches[k] += g->launches[k];
    return SIM_OK;
}

int sim_graph_kernels(const sim_graph* g, int32_t* kernels) {
    if (!g || !kernels) return SIM_ERR_NULL_PTR;
    *kernels = g->kernels;
    return SIM_OK;
}

int sim_graph_destroy(sim_graph* g) {
    if (!g) return SIM_OK;
    if (g->h) {
        cudaStreamSynchronize(g->h->last_stream);
        auto& v = g->h->graphs;
        v.erase(std::remove(v.begin(), v.end(), g), v.end());
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
    }
    delete g;
    return SIM_OK;
}

}  // extern "C"
