// sim_kernels.cu -- the fused step kernel: dynamics, collision, rewards,
// reset, field-of-view culling and ray casting of every agent of an
// environment in one CTA, step after step.  It serves the allocation-free
// single step (sim_step_static); rollouts use the split physics / render
// kernels of sim_split.cu.
//
// Work decomposition: one CTA owns one environment (all its M agents) for
// the whole horizon; CTAs pull environments from a global ticket counter in
// descending-cost order.  The environment's obstacle map is staged into
// shared memory once per environment with one cp.async.bulk.  Per step the
// CTA's warps (1) integrate and score the agents, (2) cull the map per agent
// and sensor into compact origin-relative lists, (3) cast the rays: each lane
// holds RPT rays in registers and sweeps the list, so every list entry read
// from shared memory (a broadcast) is tested against RPT rays.
#include <climits>
#include <cstdio>

#include "sim_raycast.cuh"

namespace ds {

// The fused kernel keeps one list per (agent, sensor) in arrays of lists.
__device__ inline WList fused_list(const Args& a, unsigned char* sm, int Lx) {
    WList L;
    L.sph = reinterpret_cast<float4*>(sm + a.sm.lsph) + (size_t)Lx * a.ns_max;
    L.sx = reinterpret_cast<float2*>(sm + a.sm.lr2) + (size_t)Lx * a.ns_max;
    L.box = reinterpret_cast<float4*>(sm + a.sm.lbox) + (size_t)Lx * a.nb_max * 2;
    L.cyl = nullptr;  // spheres and boxes only
    L.gat = nullptr;
    L.id = reinterpret_cast<short*>(sm + a.sm.lid) + (size_t)Lx * (a.ns_max + a.nb_max);
    L.sub = nullptr;
    L.meta = reinterpret_cast<int4*>(sm + a.sm.lmeta) + Lx;
    return L;
}

// Cull the map for every (agent, sensor) list of the CTA (one warp per list).
__device__ void build_lists(const Args& a, unsigned char* sm, const MapView& mv) {
    const int warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int L = a.M * a.S;
    const float* pose = reinterpret_cast<const float*>(sm + a.sm.pose);
    for (int Lx = warp; Lx < L; Lx += NW) {
        const float* o = pose + (Lx / a.S) * 12;
        warp_build_list<false, false>(mv, o, o + 3, a.sen[Lx % a.S], a.cull, fused_list(a, sm, Lx), cap_of(a));
    }
}

struct Item {
    int m, sidx, chunk, Lx;
};

template <int RPT>
__device__ __forceinline__ Item item_of(const Args& a, int it) {
    const int c0 = (a.sen[0].R + 32 * RPT - 1) / (32 * RPT);
    const int c1 = a.S > 1 ? (a.sen[1].R + 32 * RPT - 1) / (32 * RPT) : 0;
    const int ipa = c0 + c1;
    Item I;
    I.m = it / ipa;
    int j = it - I.m * ipa;
    I.sidx = (j >= c0) ? 1 : 0;
    I.chunk = I.sidx ? j - c0 : j;
    I.Lx = I.m * a.S + I.sidx;
    return I;
}

template <int RPT>
__device__ __forceinline__ int n_items(const Args& a) {
    const int c0 = (a.sen[0].R + 32 * RPT - 1) / (32 * RPT);
    const int c1 = a.S > 1 ? (a.sen[1].R + 32 * RPT - 1) / (32 * RPT) : 0;
    return a.M * (c0 + c1);
}

// ------------------------------------------------------- the rollout kernel
template <int RPT>
__global__ void __launch_bounds__(256, 3) k_rollout(const Args a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_env, s_flag, s_item;
    __shared__ unsigned long long s_cnt[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int M = a.M, D = a.c.D, A = a.c.A, NM = a.NM;
    const float4* prim = reinterpret_cast<const float4*>(sm + a.sm.prim);
    float* st = reinterpret_cast<float*>(sm + a.sm.st);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0ull;
    float* spre = reinterpret_cast<float*>(sm + a.sm.spre);
    float* pose = reinterpret_cast<float*>(sm + a.sm.pose);
    float* aux = reinterpret_cast<float*>(sm + a.sm.aux);
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(sm + a.sm.mbar));
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_env = atomicAdd(a.work, 1);
        __syncthreads();
        const int q = s_env;
        if (q >= a.N) break;
        const int env = a.order ? a.order[q] : q;
        const int map = a.env_map[env];
        const MapView mv = map_view(a, map, prim);
        // the shared-memory map block and cull lists are sized by the
        // capacities the caller gave: a larger map is flagged and its
        // environment left untouched (outputs unwritten, state unchanged)
        if (mv.ns > a.ns_max || mv.nb > a.nb_max || mv.nc > a.nc_max || mv.ng > a.ng_max || mv.ns < 0 ||
            mv.nb < 0) {
            if (threadIdx.x == 0) atomicOr(a.status, 4);
            __syncthreads();
            continue;
        }
        for (int i = threadIdx.x; i < M * 16; i += blockDim.x) {
            const int m = i >> 4, k = i & 15;
            st[i] = k < D ? a.state[(size_t)(env * M + m) * D + k] : 0.f;
        }
        if (!stage_map(a, sm, map, mv, phase, &s_flag)) return;
        const float drag = a.drag_env ? a.drag_env[env] : a.c.drag;
        const float lam = a.lam_env ? a.lam_env[env] : a.c.lam;
        int kpool = a.pool_k ? a.pool_k[env] : 0;
        const int T = a.render_only ? 1 : a.T;
        for (int t = 0; t < T; ++t) {
            if (!a.render_only) {
                if (a.ckpt && (t % a.K) == 0) {
                    const int c = t / a.K;
                    for (int i = threadIdx.x; i < M * D; i += blockDim.x) {
                        const int m = i / D, k = i - m * D;
                        a.ckpt[((size_t)c * NM + env * M + m) * D + k] = st[m * 16 + k];
                    }
                    if (threadIdx.x == 0) a.ckpt_k[(size_t)c * a.N + env] = kpool;
                }
                // A1: dynamics and the nearest obstacle of every agent
                for (int m = warp; m < M; m += NW) {
                    const int i = env * M + m;
                    float s[16], sp[16], act[4];
#pragma unroll
                    for (int k = 0; k < 16; ++k) s[k] = st[m * 16 + k];
#pragma unroll
                    for (int k = 0; k < 4; ++k) act[k] = k < A ? a.actions[((size_t)t * NM + i) * A + k] : 0.f;
#pragma unroll
                    for (int k = 0; k < 16; ++k) sp[k] = 0.f;
                    if (a.c.model == MODEL_RIGID) rb_step(a.c, s, act, sp);
                    else if (a.c.model == MODEL_PMD) pmd_step(a.c, s, act, sp);
                    else if (a.c.model == MODEL_SIMPLE) simple_step(a.c, s, act, sp);
                    else pm_step(a.c, drag, lam, s, act, sp);
                    float best = CUDART_INF_F;
                    int bid = -1;
                    for (int k = lane; k < mv.count(); k += 32) {
                        float d = sdf_prim(mv, k, sp);
                        if (d < best) { best = d; bid = k; }
                    }
                    warp_argmin(best, bid);
                    if (lane == 0) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) spre[m * 16 + k] = sp[k];
                        aux[m * 8 + 0] = best;
                        reinterpret_cast<int*>(aux)[m * 8 + 1] = bid;
                    }
                }
                __syncthreads();
                // A2: collisions, rewards, termination, reset, pose: one warp,
                // one lane per agent (n_agent <= 32); the reset vote is a ballot
                if (warp == 0) {
                    const int m = lane;
                    const bool on = m < M;
                    const int i = env * M + m;
                    const size_t o = (size_t)t * NM + i;
                    bool col = false;
                    if (on) {
                        const float* p = spre + m * 16;
                        const float sd = aux[m * 8 + 0];
                        col = sd < a.c.r_quad;
#pragma unroll
                        for (int k = 0; k < 3; ++k) col = col || p[k] < a.c.blo[k] || p[k] > a.c.bhi[k];
                        float pair = 0.f;
                        for (int n = 0; n < M; ++n) {
                            if (n == m) continue;
                            const float* pn = spre + n * 16;
                            float dd[3] = {p[0] - pn[0], p[1] - pn[1], p[2] - pn[2]};
                            float dij = sqrtf(dot3(dd, dd));
                            col = col || dij < a.c.d_agent;
                            float sv = relu(a.c.d_agent - dij);
                            pair += sv * sv;
                        }
                        const float* tg = a.targets + 3 * (size_t)i;
                        float e[3] = {p[0] - tg[0], p[1] - tg[1], p[2] - tg[2]};
                        float ne2 = dot3(e, e), ne = sqrtf(ne2);
                        float pos = a.c.pos_sq ? ne2 : ne;
                        float ob = (a.c.w_obs != 0.f && sd < CUDART_INF_F) ? relu(a.c.d_safe - sd) : 0.f;
                        float aa = 0.f;
                        for (int k = 0; k < A; ++k) {
                            float ak = a.actions[o * A + k];
                            aa += ak * ak;
                        }
                        float r = -a.c.w_pos * pos - a.c.w_obs * ob * ob - a.c.w_act * aa - a.c.w_agent * pair;
                        if (a.r_ctrl) a.r_ctrl[o] = r;
                        if (a.r_goal) a.r_goal[o] = (int8_t)(col ? -1 : (ne < a.c.success_radius ? 1 : 0));
                        if (a.sdf_tape) a.sdf_tape[o] = (int16_t)reinterpret_cast<int*>(aux)[m * 8 + 1];
                    }
                    const bool dn = a.c.terminate && __ballot_sync(0xffffffffu, on && col) != 0u;
                    if (on) {
                        float s[16];
                        if (dn && a.c.P > 0) {
                            const float* ps = a.pool + ((size_t)(kpool % a.c.P) * NM + i) * D;
#pragma unroll
                            for (int k = 0; k < 16; ++k) s[k] = k < D ? ps[k] : 0.f;
                        } else {
#pragma unroll
                            for (int k = 0; k < 16; ++k) s[k] = spre[m * 16 + k];
                        }
                        bool fin = true;
#pragma unroll
                        for (int k = 0; k < 16; ++k) {
                            st[m * 16 + k] = s[k];
                            fin = fin && isfinite(s[k]);
                        }
                        if (!fin) atomicOr(a.status, 1);
                        sensor_pose(a.c.model, s, pose + m * 12, pose + m * 12 + 3);
                        if (a.done) a.done[o] = dn ? 1 : 0;
                        if (a.done_tape) a.done_tape[o] = dn ? 1 : 0;
                    }
                    if (lane == 0) {
                        s_flag = dn ? 1 : 0;
                        s_item = NW;
                    }
                }
                __syncthreads();
                if (s_flag) ++kpool;
            } else {
                if (warp == 0 && lane < M) sensor_pose(a.c.model, st + lane * 16, pose + lane * 12, pose + lane * 12 + 3);
                if (threadIdx.x == 0) s_item = NW;
                __syncthreads();
            }
            if (a.S == 0) continue;
            // B: cull
            build_lists(a, sm, mv);
            __syncthreads();
            // C: rays
            const int nit = n_items<RPT>(a);
            for (int it = warp; it < nit; it = next_item(&s_item, lane)) {
                const Item I = item_of<RPT>(a, it);
                const Sensor& sen = a.sen[I.sidx];
                if (!sen.out && !sen.tape) continue;
                const float* R = pose + I.m * 12 + 3;
                const int4 meta = *(reinterpret_cast<const int4*>(sm + a.sm.lmeta) + I.Lx);
                const short* lid = reinterpret_cast<const short*>(sm + a.sm.lid) + (size_t)I.Lx * (a.ns_max + a.nb_max);
                float dx[RPT], dy[RPT], dz[RPT], tb[RPT];
                int bi[RPT];
                item_rays<RPT>(sen, R, I.chunk, lane, dx, dy, dz, tb);
#pragma unroll
                for (int r = 0; r < RPT; ++r) bi[r] = -1;
                if (meta.z < 0) cast_list<RPT, false>(fused_list(a, sm, I.Lx), meta, cap_of(a), dx, dy, dz, tb, bi);
                if (a.counters && lane == 0) {
                    const unsigned long long nr = (unsigned long long)min(32 * RPT, sen.R - I.chunk * 32 * RPT);
                    if (meta.z < 0) {
                        atomicAdd(&s_cnt[0], nr * (unsigned long long)meta.x);
                        atomicAdd(&s_cnt[1], nr * (unsigned long long)meta.y);
                    }
                    atomicAdd(&s_cnt[2], nr);
                }
                const size_t base = ((size_t)t * NM + env * M + I.m) * sen.R;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int ray = I.chunk * 32 * RPT + r * 32 + lane;
                    if (ray >= sen.R) continue;
                    float v;
                    int id;
                    if (meta.z >= 0) { v = 0.f; id = meta.z; }
                    else if (bi[r] < 0) { v = sen.range; id = -1; }
                    else {
                        v = fminf(sen.kind == 0 ? tb[r] * __ldg(&sen.dir[ray].w) : tb[r], sen.range);
                        id = lid[bi[r]];
                    }
                    if (sen.out) sen.out[base + ray] = v;
                    if (sen.tape) sen.tape[base + ray] = (int16_t)id;
                }
            }
        }
        __syncthreads();
        if (!a.render_only) {
            for (int i = threadIdx.x; i < M * D; i += blockDim.x) {
                const int m = i / D, k = i - m * D;
                a.state[(size_t)(env * M + m) * D + k] = st[m * 16 + k];
            }
            if (threadIdx.x == 0 && a.pool_k) a.pool_k[env] = kpool;
            if (threadIdx.x == 0) s_cnt[3] += (unsigned long long)T;
        }
    }
    __syncthreads();
    if (a.counters && threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(a.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

// ------------------------------------------------------------ launchers
template <int RPT>
static cudaError_t launch_rpt(const Args& a, int grid, int block, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_rollout<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rollout<RPT><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int RPT>
static cudaError_t occupancy_rpt(int block, size_t smem, int* n) {
    cudaError_t e = cudaFuncSetAttribute(k_rollout<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_rollout<RPT>, block, smem);
}

bool rpt_supported(int rpt) {
    return rpt == 1 || rpt == 2 || rpt == 3 || rpt == 4 || rpt == 5 || rpt == 6 || rpt == 8;
}

cudaError_t launch_fused(int rpt, const Args& a, int grid, int block, size_t smem, cudaStream_t st) {
    switch (rpt) {
        case 1: return launch_rpt<1>(a, grid, block, smem, st);
        case 2: return launch_rpt<2>(a, grid, block, smem, st);
        case 3: return launch_rpt<3>(a, grid, block, smem, st);
        case 4: return launch_rpt<4>(a, grid, block, smem, st);
        case 5: return launch_rpt<5>(a, grid, block, smem, st);
        case 6: return launch_rpt<6>(a, grid, block, smem, st);
        case 8: return launch_rpt<8>(a, grid, block, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_fused(int rpt, int block, size_t smem, int* n) {
    switch (rpt) {
        case 1: return occupancy_rpt<1>(block, smem, n);
        case 2: return occupancy_rpt<2>(block, smem, n);
        case 3: return occupancy_rpt<3>(block, smem, n);
        case 4: return occupancy_rpt<4>(block, smem, n);
        case 5: return occupancy_rpt<5>(block, smem, n);
        case 6: return occupancy_rpt<6>(block, smem, n);
        case 8: return occupancy_rpt<8>(block, smem, n);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ds
