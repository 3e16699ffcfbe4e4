// sim_static.cu -- sim_step_static: one environment step that allocates no
// device memory.  It serves callers that cannot call cudaMalloc (for
// example code running inside a memory pool or arena owned by another
// framework, or a process whose device allocations are fixed up front):
// they pass every input and output buffer, and the few scratch words and ray
// tables the step needs live in one file-scope device array that every GPU
// which loads the library holds until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "diffsim.h"
#include "sim_kernels.cuh"

namespace ds {
bool rpt_supported(int rpt);
cudaError_t launch_fused(int rpt, const Args& a, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t occupancy_fused(int rpt, int block, size_t smem, int* n);
}  // namespace ds

namespace {

// Scratch layout: [0, 64) control words (work ticket, status, 4 counters),
// then the camera and LiDAR ray tables (float4 per ray), then their clamp
// distances (float per ray).
constexpr size_t kScratchBytes = SIM_STATIC_SCRATCH_BYTES;
constexpr size_t kCtrlBytes = 64;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device ordinal: the scratch address and the id of the context it was
// looked up in.  A device's context can be torn down and made again
// (cudaDeviceReset), which reloads the module at a new address; the context
// id tells the cached address apart from a stale one.
unsigned char* g_ptr[kMaxDevices] = {nullptr};
unsigned long long g_ctx[kMaxDevices] = {0};

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrent g_get_ctx = nullptr;
CtxGetId g_get_id = nullptr;
bool g_looked_up = false;

// Id of the calling thread's current context, 0 if none or unknown.  The
// driver functions come through the runtime's entry-point query, so the
// library needs no link against the driver library.
unsigned long long current_ctx_id() {
    if (!g_looked_up) {
        g_looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_get_ctx = reinterpret_cast<CtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_get_id = reinterpret_cast<CtxGetId>(f);
        cudaGetLastError();
    }
    if (!g_get_ctx || !g_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_scratch on the current device: looked up once per
// device and context (again after the device's context was reset; on every
// call if the context id cannot be read).
int scratch_ptr(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return SIM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_ptr[dev] || id == 0 || id != g_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return SIM_ERR_CUDA;
        }
        g_ptr[dev] = static_cast<unsigned char*>(p);
        g_ctx[dev] = current_ctx_id();  // the lookup made the device's context current
    }
    *out = g_ptr[dev];
    return SIM_OK;
}

// Body-frame ray directions (x, y, z) and output factor w, in double then
// rounded, with the same camera and LiDAR models as sim_create.
__global__ void k_fill_rays(float4* cam, float* cam_t, int W, int H, double th, double range_c, float4* lid,
                            float* lid_t, int C, int Az, double el_lo, double el_hi, float range_l) {
    const int Rc = W * H, Rl = C * Az;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < Rc + Rl; r += gridDim.x * blockDim.x) {
        if (r < Rc) {
            const int j = r / W, i = r - j * W;
            const double tv = th * H / W;
            const double u = (2.0 * (i + 0.5) / W - 1.0) * th, v = (2.0 * (j + 0.5) / H - 1.0) * tv;
            const double n = sqrt(1.0 + u * u + v * v);
            cam[r] = make_float4((float)(1.0 / n), (float)(-u / n), (float)(-v / n), (float)(1.0 / n));
            cam_t[r] = (float)(range_c * n);
        } else {
            const int q = r - Rc, ch = q / Az, k = q - ch * Az;
            const double el = C > 1 ? el_lo + ch * (el_hi - el_lo) / (C - 1) : 0.5 * (el_lo + el_hi);
            const double az = 2.0 * M_PI * k / Az;
            lid[q] = make_float4((float)(cos(el) * cos(az)), (float)(cos(el) * sin(az)), (float)sin(el), 1.f);
            lid_t[q] = range_l;
        }
    }
}

bool bad_cfg(const sim_config* c) {
    if (c->model < SIM_MODEL_POINT_MASS || c->model > SIM_MODEL_SIMPLE) return true;
    if (c->n_env < 1 || c->n_agent < 1 || c->n_agent > 32) return true;
    if (!(c->dt > 0.f) || !std::isfinite(c->dt)) return true;
    if (c->cam_w < 0 || c->cam_h < 0 || c->lid_ch < 0 || c->lid_az < 0) return true;
    if (c->cam_w > 0 && (c->cam_h < 1 || !(c->cam_hfov > 0.f && c->cam_hfov < 3.1f) || !(c->cam_range > 0.f)))
        return true;
    if (c->lid_ch > 0 && (c->lid_az < 1 || !(c->lid_range > 0.f) || !(c->lid_elev_lo <= c->lid_elev_hi)))
        return true;
    if (c->model == SIM_MODEL_RIGID)
        for (int i = 0; i < 3; ++i)
            if (!(c->inertia[i] > 0.f)) return true;
    if (c->model == SIM_MODEL_RIGID && !(c->mass > 0.f)) return true;
    if (c->pool_size < 0 || c->cull < -1 || c->cull > 2) return true;
    if (c->warps_per_cta < 0 || c->warps_per_cta > 8) return true;
    if (c->rays_per_thread != 0 && !ds::rpt_supported(c->rays_per_thread)) return true;
    if (c->task != SIM_TASK_REACH) return true;  // the reaching task only
    return false;
}

size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

extern "C" int sim_step_static(const sim_config* cfg, const float* prims, const int32_t* map_off,
                               const int32_t* map_ns, const int32_t* map_nb, int32_t ns_max, int32_t nb_max,
                               const int32_t* env_map, const float* targets, const float* pool, float* state,
                               const float* actions, float* depth, float* lidar, float* r_ctrl, int8_t* r_goal,
                               uint8_t* done, int32_t* pool_k, int32_t* status, sim_stream_t stream) {
    if (!cfg || !map_off || !map_ns || !map_nb || !env_map || !targets || !state || !actions)
        return SIM_ERR_NULL_PTR;
    if (bad_cfg(cfg)) return SIM_ERR_INVALID_ARG;
    if (ns_max < 0 || nb_max < 0 || ns_max + nb_max > 32767) return SIM_ERR_SIZE;
    if (ns_max + nb_max > 0 && !prims) return SIM_ERR_NULL_PTR;
    if (cfg->terminate && cfg->pool_size > 0 && !pool) return SIM_ERR_NULL_PTR;
    const int Rc = cfg->cam_w > 0 ? cfg->cam_w * cfg->cam_h : 0;
    const int Rl = cfg->lid_ch > 0 ? cfg->lid_ch * cfg->lid_az : 0;
    // the ray tables must fit the static scratch next to the control words
    if (kCtrlBytes + 20 * ((size_t)Rc + Rl) > kScratchBytes) return SIM_ERR_SIZE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return SIM_ERR_CUDA;
    unsigned char* base = nullptr;
    int rc = scratch_ptr(dev, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    ds::Args a;
    memset(&a, 0, sizeof(a));
    const sim_config& c = *cfg;
    a.c.model = c.model; a.c.M = c.n_agent; a.c.D = sim_state_dim(c.model);
    a.c.A = sim_action_dim(c.model);
    a.c.dt = c.dt; a.c.g = c.gravity; a.c.lam = c.lam; a.c.drag = c.drag;
    a.c.act_scale = c.act_scale; a.c.ema_alpha = c.ema_alpha; a.c.mass = c.mass;
    for (int i = 0; i < 3; ++i) {
        a.c.J[i] = c.inertia[i]; a.c.K[i] = c.k_rate[i]; a.c.Dd[i] = c.drag_body[i];
        a.c.rs[i] = c.rate_scale[i]; a.c.blo[i] = c.bound_lo[i]; a.c.bhi[i] = c.bound_hi[i];
    }
    a.c.pos_sq = c.pos_sq; a.c.w_pos = c.w_pos; a.c.w_obs = c.w_obs; a.c.d_safe = c.d_safe;
    a.c.w_act = c.w_act; a.c.w_agent = c.w_agent; a.c.d_agent = c.d_agent;
    a.c.success_radius = c.success_radius; a.c.r_quad = c.r_quad;
    a.c.terminate = c.terminate; a.c.P = pool ? c.pool_size : 0;
    a.N = c.n_env; a.M = c.n_agent; a.NM = c.n_env * c.n_agent; a.T = 1; a.K = 1;
    a.ns_max = ns_max; a.nb_max = nb_max; a.cull = c.cull;
    // sensors: tables in scratch, same models and culling constants as sim_create
    float4* cam = reinterpret_cast<float4*>(base + kCtrlBytes);
    float4* lid = cam + Rc;
    float* cam_t = reinterpret_cast<float*>(lid + Rl);
    float* lid_t = cam_t + Rc;
    int S = 0;
    if (Rc) {
        const double th = std::tan(0.5 * (double)c.cam_hfov), tv = th * c.cam_h / c.cam_w;
        const double u = (1.0 - 1.0 / c.cam_w) * th, v = (1.0 - 1.0 / c.cam_h) * tv;
        const double fmin = 1.0 / std::sqrt(1.0 + u * u + v * v);
        ds::Sensor& s = a.sen[S++];
        s.R = Rc; s.dir = cam; s.tmax = cam_t; s.range = c.cam_range; s.kind = 0;
        s.c0 = (float)th; s.c1 = (float)tv;
        s.c2 = (float)(1.0 / std::sqrt(1.0 + th * th)); s.c3 = (float)(1.0 / std::sqrt(1.0 + tv * tv));
        s.maxlen = (float)(c.cam_range / fmin);
        s.out = depth;
    }
    if (Rl) {
        ds::Sensor& s = a.sen[S++];
        s.R = Rl; s.dir = lid; s.tmax = lid_t; s.range = c.lid_range; s.kind = 1;
        s.c0 = c.lid_elev_lo; s.c1 = c.lid_elev_hi; s.maxlen = c.lid_range;
        s.out = lidar;
    }
    a.S = S;
    a.prims = reinterpret_cast<const float4*>(prims);
    a.map_off = map_off; a.map_ns = map_ns; a.map_nb = map_nb;
    a.env_map = env_map; a.order = nullptr; a.targets = targets; a.pool = pool;
    a.state = state; a.actions = actions; a.pool_k = pool_k;
    a.r_ctrl = r_ctrl; a.r_goal = r_goal; a.done = done;
    a.work = reinterpret_cast<int*>(base);
    a.status = reinterpret_cast<int*>(base) + 1;
    a.counters = reinterpret_cast<unsigned long long*>(base + 16);
    // shared-memory layout of the forward kernel (map block, cull lists, per-agent rows)
    const int M = c.n_agent, L = M * S;
    size_t o = 0;
    auto take = [&](int& f, size_t bytes) { f = (int)o; o = a16(o + bytes); };
    take(a.sm.prim, (size_t)(ns_max + 2 * nb_max) * 16);
    take(a.sm.lsph, (size_t)L * ns_max * 16);
    take(a.sm.lbox, (size_t)L * nb_max * 32);
    take(a.sm.lr2, (size_t)L * ns_max * 8);
    take(a.sm.lid, (size_t)L * (ns_max + nb_max) * 2);
    take(a.sm.lmeta, (size_t)L * 16);
    take(a.sm.st, (size_t)M * 64);
    take(a.sm.spre, (size_t)M * 64);
    take(a.sm.pose, (size_t)M * 48);
    take(a.sm.aux, (size_t)M * 32);
    take(a.sm.mbar, 16);
    a.sm.total = (int)o;
    int maxsm = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SIM_ERR_CUDA;
    if (a.sm.total > maxsm) return SIM_ERR_SIZE;
    const int nw = c.warps_per_cta ? c.warps_per_cta : 8;
    const int rpt = c.rays_per_thread ? c.rays_per_thread : 4;
    int occ = 0;
    if (ds::occupancy_fused(rpt, 32 * nw, a.sm.total, &occ) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return SIM_ERR_UNSUPPORTED;
    }
    const int grid = (int)std::min<long>((long)occ * nsm, c.n_env);
    // every call rewrites its control words and ray tables (the array keeps
    // the previous call's contents)
    if (cudaMemsetAsync(base, 0, kCtrlBytes, st) != cudaSuccess) return SIM_ERR_CUDA;
    if (Rc + Rl) {
        k_fill_rays<<<(Rc + Rl + 255) / 256, 256, 0, st>>>(cam, cam_t, c.cam_w, c.cam_h,
                                                           std::tan(0.5 * (double)c.cam_hfov), (double)c.cam_range,
                                                           lid, lid_t, c.lid_ch, c.lid_az, c.lid_elev_lo,
                                                           c.lid_elev_hi, c.lid_range);
        if (cudaGetLastError() != cudaSuccess) return SIM_ERR_CUDA;
    }
    e = ds::launch_fused(rpt, a, grid, 32 * nw, a.sm.total, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SIM_ERR_CUDA;
    }
    // this call's status word (the control words were cleared above)
    if (status && cudaMemcpyAsync(status, a.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return SIM_ERR_CUDA;
    return SIM_OK;
}
