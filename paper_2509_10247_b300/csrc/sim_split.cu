// sim_split.cu -- rollout and adjoint as two kernels each.
//
// The sequential part of a step (dynamics Eq. 1 / Eq. 3, collisions,
// rewards, termination and reset, sensor pose; Sec. III-A to III-D) is light
// and latency-bound; the ray casting of Sec. III-B is heavy and has no
// dependence between steps once the poses are known (actions are inputs).
// So the physics runs first, one warp per environment with one lane per
// agent and the state in registers for the whole horizon, writing the pose
// trajectory [T][NM][12] (origin, rotation); then every (step, agent,
// sensor) is rendered independently by one warp that culls the map into its
// own shared-memory list and sweeps its rays.  The adjoint (Eq. 5) mirrors
// it: per (step, agent) ray cotangents reduce to a pose cotangent, then the
// physics is reverted environment by environment from checkpoints.
#include "sim_raycast.cuh"

namespace ds {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void load_row(const float* src, int D, bool on, int model, float* s) {
#pragma unroll
    for (int k = 0; k < 16; ++k) s[k] = (on && k < D) ? src[k] : 0.f;
    if (!on && model == MODEL_RIGID) s[3] = 1.f;  // a harmless unit quaternion on idle lanes
    if (!on && model == MODEL_SIMPLE) s[6] = s[10] = s[14] = 1.f;  // and rotation
}

__device__ __forceinline__ void step_agent(const Phys& c, float drag, float lam, const float* s, const float* act,
                                           float* sp) {
#pragma unroll
    for (int k = 0; k < 16; ++k) sp[k] = 0.f;
    if (c.model == MODEL_RIGID) rb_step(c, s, act, sp);
    else if (c.model == MODEL_PMD) pmd_step(c, s, act, sp);
    else if (c.model == MODEL_SIMPLE) simple_step(c, s, act, sp);
    else pm_step(c, drag, lam, s, act, sp);
}

// Nearest obstacle of every agent of the warp's environment: the warp splits
// into groups of G = 32 / M' lanes (M' = M rounded up to a power of two),
// group g scans the map for agent g at position p (lane g's p), then lane m
// receives agent m's signed distance and arg-min (lowest id among ties).
__device__ __forceinline__ void nearest_obstacle(const MapView& mv, int M, const float* p, float& sd, int& id) {
    const int lane = threadIdx.x & 31;
    int Mp = 1;
    while (Mp < M) Mp <<= 1;
    const int G = 32 / Mp;
    const int gm = lane / G, gl = lane - gm * G;
    const float q[3] = {__shfl_sync(0xffffffffu, p[0], gm), __shfl_sync(0xffffffffu, p[1], gm),
                        __shfl_sync(0xffffffffu, p[2], gm)};
    float best = CUDART_INF_F;
    int bid = -1;
    if (gm < M) {
        // one loop per kind, two primitives in flight; a lane visits its ids
        // in increasing order and keeps the first of equal distances
        const int ns = mv.ns, nb = mv.nb, np = mv.count();
        int k = gl;
        for (; k + 3 * G < ns; k += 4 * G) {
            const float d0 = sdf_sphere(mv.prim[k], q), d1 = sdf_sphere(mv.prim[k + G], q);
            const float d2 = sdf_sphere(mv.prim[k + 2 * G], q), d3 = sdf_sphere(mv.prim[k + 3 * G], q);
            if (d0 < best) { best = d0; bid = k; }
            if (d1 < best) { best = d1; bid = k + G; }
            if (d2 < best) { best = d2; bid = k + 2 * G; }
            if (d3 < best) { best = d3; bid = k + 3 * G; }
        }
        for (; k < ns; k += G) {
            const float d0 = sdf_sphere(mv.prim[k], q);
            if (d0 < best) { best = d0; bid = k; }
        }
        int j = gl;
        for (; j + G < nb; j += 2 * G) {
            const float d0 = sdf_box_lohi(mv.box(j)[0], mv.box(j)[1], q);
            const float d1 = sdf_box_lohi(mv.box(j + G)[0], mv.box(j + G)[1], q);
            if (d0 < best) { best = d0; bid = ns + j; }
            if (d1 < best) { best = d1; bid = ns + j + G; }
        }
        if (j < nb) {
            const float d0 = sdf_box_lohi(mv.box(j)[0], mv.box(j)[1], q);
            if (d0 < best) { best = d0; bid = ns + j; }
        }
        for (int c = ns + nb + gl; c < np; c += G) {  // cylinders and gates
            const float d = sdf_prim(mv, c, q);
            if (d < best) { best = d; bid = c; }
        }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bid, o);
        if (v2 < best || (v2 == best && (unsigned)i2 < (unsigned)bid)) { best = v2; bid = i2; }
    }
    const int src = lane < Mp ? lane * G : 0;
    sd = __shfl_sync(0xffffffffu, best, src);
    id = __shfl_sync(0xffffffffu, bid, src);
}

// The same search by one lane for its own position over the whole map (the
// lanes of a warp may belong to different environments).
__device__ __forceinline__ void nearest_obstacle_lane(const MapView& mv, const float* q, float& sd, int& id) {
    float best = CUDART_INF_F;
    int bid = -1;
    const int ns = mv.ns, nb = mv.nb, np = mv.count();
    for (int k = 0; k < ns; ++k) {
        const float d = sdf_sphere(mv.prim[k], q);
        if (d < best) { best = d; bid = k; }
    }
    for (int j = 0; j < nb; ++j) {
        const float d = sdf_box_lohi(mv.box(j)[0], mv.box(j)[1], q);
        if (d < best) { best = d; bid = ns + j; }
    }
    for (int c = ns + nb; c < np; ++c) {
        const float d = sdf_prim(mv, c, q);
        if (d < best) { best = d; bid = c; }
    }
    sd = best;
    id = bid;
}

__host__ __device__ inline int pow2_ceil(int m) {
    int p = 1;
    while (p < m) p <<= 1;
    return p;
}

// Environments per warp of the physics adjoint: the warp's lanes form groups
// of pow2_ceil(M) lanes, one environment per group and a lane per agent, as
// many groups as fit in 32 lanes and in 96 KiB of segment states.
__host__ __device__ inline int phys_bwd_envs_per_warp(int K, int M) {
    const size_t per_env = (size_t)(K + 1) * M * 16 * sizeof(float);
    int E = 32 / pow2_ceil(M);
    while (E > 1 && (size_t)E * per_env > 96 * 1024) E >>= 1;
    return E;
}

// ----------------------------------------------------------- forward physics
// A warp holds 32 / pow2_ceil(M) environments, a lane group per environment
// and a lane per agent; environments are taken in the work order (grouped
// by map, so a warp's groups scan maps of one size).  render_only: write the
// pose of the current state at step 0 and return.
// EXT: the racing task or the IMU readout is on (else their code is compiled out).
template <bool EXT>
__global__ void __launch_bounds__(128) k_physics(const Args a) {
    const int lane = threadIdx.x & 31;
    const int M = a.M, D = a.c.D, A = a.c.A, NM = a.NM;
    const int Mp = pow2_ceil(M), E = 32 / Mp;
    const int grp = lane / Mp, agent = lane - grp * Mp, gbase = grp * Mp;
    const unsigned gmask = Mp == 32 ? 0xffffffffu : ((1u << Mp) - 1u) << gbase;
    const int q0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * E;
    if (q0 >= a.N) return;
    const bool live = q0 + grp < a.N;
    const int q = live ? q0 + grp : q0;
    const int env = a.order ? a.order[q] : q;  // idle groups read a valid environment, write nothing
    const int map = a.env_map[env];
    const MapView mv = map_view(a, map, a.prims + a.map_off[map]);
    const bool on = live && agent < M;
    const int i = env * M + (on ? agent : 0);
    const float drag = a.drag_env ? a.drag_env[env] : a.c.drag;
    const float lam = a.lam_env ? a.lam_env[env] : a.c.lam;
    float s[16];
    load_row(a.state + (size_t)i * D, D, on, a.c.model, s);
    if (a.render_only) {
        if (on && a.poses) sensor_pose(a.c.model, s, a.poses + (size_t)i * 12, a.poses + (size_t)i * 12 + 3);
        return;
    }
    int kpool = a.pool_k ? a.pool_k[env] : 0;
    const bool racing = EXT && a.c.task == 1;
    const bool imu = EXT && a.imu;
    int gk = (racing && on) ? a.gate_k[i] : 0;
    float bias[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) bias[k] = (imu && a.imu_noise && on) ? a.imu_bias[(size_t)i * 6 + k] : 0.f;
    for (int t = 0; t < a.T; ++t) {
        const size_t o = (size_t)t * NM + i;
        if (a.ckpt && (t % a.K) == 0) {
            const int c = t / a.K;
            if (on)
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < D) a.ckpt[((size_t)c * NM + i) * D + k] = s[k];
            if (live && agent == 0) a.ckpt_k[(size_t)c * a.N + env] = kpool;
        }
        float act[4], sp[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) act[k] = (on && k < A) ? a.actions[o * A + k] : 0.f;
        step_agent(a.c, drag, lam, s, act, sp);
        float sd;
        int bid;
        if (E > 1) nearest_obstacle_lane(mv, sp, sd, bid);
        else nearest_obstacle(mv, M, sp, sd, bid);
        // collisions and the dense / sparse rewards (Sec. III-C, III-E)
        bool col = sd < a.c.r_quad;
#pragma unroll
        for (int k = 0; k < 3; ++k) col = col || sp[k] < a.c.blo[k] || sp[k] > a.c.bhi[k];
        float pair = 0.f;
        for (int n = 0; n < M; ++n) {
            const float px = __shfl_sync(0xffffffffu, sp[0], gbase + n),
                        py = __shfl_sync(0xffffffffu, sp[1], gbase + n),
                        pz = __shfl_sync(0xffffffffu, sp[2], gbase + n);
            if (n == agent) continue;
            const float dd[3] = {sp[0] - px, sp[1] - py, sp[2] - pz};
            const float dij = sqrtf(dot3(dd, dd));
            col = col || dij < a.c.d_agent;
            const float sv = relu(a.c.d_agent - dij);
            pair += sv * sv;
        }
        const bool dn = a.c.terminate && (__ballot_sync(0xffffffffu, on && col) & gmask) != 0u;
        if (on) {
            const float ob = (a.c.w_obs != 0.f && sd < CUDART_INF_F) ? relu(a.c.d_safe - sd) : 0.f;
            float aa = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < A) aa += act[k] * act[k];
            const float rest = -a.c.w_obs * ob * ob - a.c.w_act * aa - a.c.w_agent * pair;
            if (racing) {
                // progress towards the targeted gate; +1 for passing it
                const float4 g0 = mv.gate(gk)[0], g1 = mv.gate(gk)[1];
                const float e0[3] = {s[0] - g0.x, s[1] - g0.y, s[2] - g0.z};
                const float e1[3] = {sp[0] - g0.x, sp[1] - g0.y, sp[2] - g0.z};
                const bool passed = gate_passed(g0, g1, s, sp);
                if (a.r_ctrl) a.r_ctrl[o] = a.c.w_pos * (sqrtf(dot3(e0, e0)) - sqrtf(dot3(e1, e1))) + rest;
                if (a.r_goal) a.r_goal[o] = (int8_t)(col ? -1 : (passed ? 1 : 0));
                if (a.gate_tape) a.gate_tape[o] = (int16_t)gk;
                if (passed) gk = gk + 1 < mv.ng ? gk + 1 : 0;
            } else {
                const float* tg = a.targets + 3 * (size_t)i;
                const float e[3] = {sp[0] - tg[0], sp[1] - tg[1], sp[2] - tg[2]};
                const float ne2 = dot3(e, e), ne = sqrtf(ne2);
                const float pos = a.c.pos_sq ? ne2 : ne;
                if (a.r_ctrl) a.r_ctrl[o] = -a.c.w_pos * pos + rest;
                if (a.r_goal) a.r_goal[o] = (int8_t)(col ? -1 : (ne < a.c.success_radius ? 1 : 0));
            }
            if (a.sdf_tape) a.sdf_tape[o] = (int16_t)bid;
            if (a.done) a.done[o] = dn ? 1 : 0;
            if (a.done_tape) a.done_tape[o] = dn ? 1 : 0;
        }
        float imu6[6];
        if (imu && on && !dn) imu_eval(a.c, drag, s, act, sp, imu6);
        // termination and reset of the whole environment from the pool
        if (dn && a.c.P > 0) load_row(a.pool + ((size_t)(kpool % a.c.P) * NM + i) * D, D, on, a.c.model, s);
        else {
#pragma unroll
            for (int k = 0; k < 16; ++k) s[k] = sp[k];
        }
        if (dn) {
            ++kpool;
            gk = 0;
        }
        if (imu && on) {
            if (dn) imu_reset(a.c, s, imu6);
            if (a.imu_noise) {
                const float* z = a.imu_noise + o * 12;
                const float sdt = sqrtf(a.c.dt);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    if (dn) bias[k] = 0.f;
                    imu6[k] += fmaf(a.c.imu_noise[k / 3], z[k], bias[k]);
                    bias[k] = fmaf(a.c.imu_walk[k / 3] * sdt, z[6 + k], bias[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) a.imu[o * 6 + k] = imu6[k];
        }
        if (on) {
            bool fin = true;
#pragma unroll
            for (int k = 0; k < 16; ++k) fin = fin && isfinite(s[k]);
            if (!fin) atomicOr(a.status, 1);
            if (a.poses) sensor_pose(a.c.model, s, a.poses + o * 12, a.poses + o * 12 + 3);
        }
    }
    if (on)
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < D) a.state[(size_t)i * D + k] = s[k];
    if (live && agent == 0 && a.pool_k) a.pool_k[env] = kpool;
    if (racing && on) a.gate_k[i] = gk;
    if (imu && a.imu_noise && on)
#pragma unroll
        for (int k = 0; k < 6; ++k) a.imu_bias[(size_t)i * 6 + k] = bias[k];
}

// ------------------------------------------------------------------ render
// Persistent CTAs take environments from a ticket (descending work); the
// environment's map is staged once into shared memory; its T x M x S items
// (step, agent, sensor) are taken by warps from a CTA ticket.  A warp culls
// the map into its private list and sweeps all rays of the item.
// Rays of chunks [c0, c1) of one (step, agent, sensor) item against its
// cull list L (meta: its counts): cast, count, write depth / range and the
// hit tape.  One full warp.
template <int RPT, bool EXTRA, bool CASTW = false>
__device__ __forceinline__ void render_chunks(const Args& a, const WList& L, const int4& meta, const LCap& cap,
                                              const Sensor& sen, const float* R, int c0, int c1, size_t base,
                                              unsigned long long* s_cnt) {
    const int lane = threadIdx.x & 31;
    float* const outp = sen.out ? sen.out + base : nullptr;
    int16_t* const tapep = sen.tape ? sen.tape + base : nullptr;
    for (int ch = c0; ch < c1; ++ch) {
        float dx[RPT], dy[RPT], dz[RPT], tb[RPT];
        int bi[RPT];
        item_rays<RPT>(sen, R, ch, lane, dx, dy, dz, tb);
#pragma unroll
        for (int r = 0; r < RPT; ++r) bi[r] = -1;
        int4 nsub = make_int4(meta.x, meta.y, meta.w & 0xffff, meta.w >> 16);
        if (meta.z < 0) {
            if (CASTW) {
                const bool sub = a.cull > 1 && sen.cone;
                if (sub) nsub = chunk_slots<EXTRA>(L, meta, cap, sen, a.cull, ch, R);
                cast_warp_per_ray<RPT>(L, nsub, cap, sub, dx, dy, dz, tb, bi);
            } else if (a.cull > 1 && sen.cone) {
                nsub = chunk_slots<EXTRA>(L, meta, cap, sen, a.cull, ch, R);
                cast_sub<RPT, EXTRA>(L, nsub, cap, dx, dy, dz, tb, bi);
            } else {
                cast_list<RPT, EXTRA>(L, meta, cap, dx, dy, dz, tb, bi);
            }
        }
        if (a.counters && lane == 0) {
            const unsigned long long nr = (unsigned long long)min(32 * RPT, sen.R - ch * 32 * RPT);
            if (meta.z < 0) {
                atomicAdd(&s_cnt[0], nr * (unsigned long long)nsub.x);
                atomicAdd(&s_cnt[1], nr * (unsigned long long)(nsub.y + nsub.z + nsub.w));
            }
            atomicAdd(&s_cnt[2], nr);
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int j = ch * 32 * RPT + r * 32 + lane;
            if (j >= sen.R) continue;
            const int ray = out_index(sen, j);
            float v;
            int id;
            if (meta.z >= 0) { v = 0.f; id = -2; }  // origin inside a primitive: no ray cotangent
            else if (bi[r] < 0) { v = sen.range; id = -1; }
            else {
                v = fminf(sen.kind == 0 ? tb[r] * __ldg(&sen.dir[j].w) : tb[r], sen.range);
                id = L.id[bi[r]];
            }
            if (outp) outp[ray] = v;
            if (tapep) tapep[ray] = (int16_t)id;
        }
    }
}

// CASTW: warp per ray (cast_mode 1, maps of spheres and boxes), compiled apart
// so that the thread-per-ray kernels keep their registers.
// ONE: a single sensor (index 0, known at compile time: its fields are
// kernel-parameter operands instead of loads indexed by the item's sensor).
template <int RPT, bool EXTRA, bool COOP, bool CASTW = false, bool ONE = false>
__global__ void __launch_bounds__(256, 4) k_render(const Args a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_env, s_flag, s_item;
    __shared__ unsigned long long s_cnt[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int M = a.M, S = a.S, NM = a.NM;
    const float4* prim = reinterpret_cast<const float4*>(sm + a.sm.prim);
    const LCap cap = cap_of(a);
    const WList L = wlist_at(sm + a.sm.wlist + (size_t)warp * a.sm.wstride, cap);
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(sm + a.sm.mbar));
    __syncthreads();
    uint32_t phase = 0;
    // items: (step, agent, sensor, part); a sensor's chunks are split into
    // rparts consecutive ranges so that short horizons still give every warp
    // of the CTA work
    const int nch0 = (a.sen[0].R + 32 * RPT - 1) / (32 * RPT);
    const int nch1 = S > 1 ? (a.sen[1].R + 32 * RPT - 1) / (32 * RPT) : 0;
    const int P0 = S > 0 ? min(a.rparts[0], max(nch0, 1)) : 0, P1 = S > 1 ? min(a.rparts[1], max(nch1, 1)) : 0;
    const int per_tm = P0 + P1;
    const int per_env = a.T * M * per_tm;
    // few (step, agent, sensor) lists split into parts: each list is built
    // once per environment, by its own warp, and shared by the warps that
    // cast its parts (each keeps its chunk sub-lists in its own region)
    const int nlists = a.T * M * S;
    const bool coop = COOP && per_tm > S && nlists <= NW;
    for (;;) {
        if (threadIdx.x == 0) {
            s_env = atomicAdd(a.work, 1);
            s_item = NW;
        }
        __syncthreads();
        const int q = s_env;
        if (q >= a.N) break;
        const int env = a.order ? a.order[q] : q;
        const int map = a.env_map[env];
        const MapView mv = map_view(a, map, prim);
        if (!stage_map(a, sm, map, mv, phase, &s_flag)) return;
        prep_boxes(sm, a, mv.ns, mv.nb);
        if (coop) {
            if (warp < nlists) {
                const int tm = warp / S, si = warp - tm * S, t = tm / M, m = tm - t * M;
                const Sensor& sen = a.sen[si];
                if (sen.out || sen.tape) {
                    const size_t ti = (size_t)t * NM + env * M + m;
                    float o[3], R[9];
                    load_pose(a.poses + ti * 12, o, R);
                    warp_build_list<EXTRA, true>(mv, o, R, sen, a.cull, L, cap);
                }
            }
            __syncthreads();
        }
        const int lgM = (M & (M - 1)) == 0 ? __ffs(M) - 1 : -1;  // M a power of two: shifts
        for (int it = warp; it < per_env; it = next_item(&s_item, lane)) {
            const int tm = per_tm == 1 ? it : div_small(it, per_tm), r = it - tm * per_tm;
            const int t = lgM >= 0 ? tm >> lgM : div_small(tm, M), m = tm - t * M;
            const int si = r < P0 ? 0 : 1, part = si ? r - P0 : r, np = si ? P1 : P0, nchs = si ? nch1 : nch0;
            const int c0 = np == 1 ? 0 : div_small(part * nchs, np), c1 = np == 1 ? nchs : div_small((part + 1) * nchs, np);
            auto item = [&](const Sensor& sen) {
                if (!sen.out && !sen.tape) return;
                const size_t ti = (size_t)t * NM + env * M + m;
                float o[3], R[9];
                load_pose(a.poses + ti * 12, o, R);
                const size_t base = ti * sen.R;
                int4 meta;
                WList Lv = L;
                if (coop) {  // the item's list, built by warp (tm * S + si) in this environment's first phase
                    Lv = wlist_at(sm + a.sm.wlist + (size_t)(tm * S + si) * a.sm.wstride, cap);
                    Lv.sub = L.sub;
                    meta = *Lv.meta;
                } else {
                    meta = warp_build_list<EXTRA, true>(mv, o, R, sen, a.cull, L, cap);
                }
                render_chunks<RPT, EXTRA, CASTW>(a, Lv, meta, cap, sen, R, c0, c1, base, s_cnt);
            };
            if (ONE) item(a.sen[0]);
            else item(a.sen[si]);
            __syncwarp();
        }
        if (threadIdx.x == 0) s_cnt[3] += (unsigned long long)(a.T);
        __syncthreads();
    }
    __syncthreads();
    if (a.counters && threadIdx.x < 4 && s_cnt[threadIdx.x]) atomicAdd(a.counters + threadIdx.x, s_cnt[threadIdx.x]);
}

// ------------------------------------------------------ render from hits
// Depth / range of the current poses from recorded hit ids (sen.tape read,
// sen.out written): a CTA per agent (grid-stride), a thread per ray slot,
// each evaluating only its recorded primitive with the cast's own entry and
// test (hit_distance), so the image equals a full render of the same state
// bit for bit.  Ids: -1 miss (range), -2 origin inside a primitive (0); ids
// outside the map are treated as misses.
template <bool EXTRA>
__global__ void __launch_bounds__(256) k_render_hits(const Args a) {
    const int R0 = a.sen[0].R, Rt = R0 + (a.S > 1 ? a.sen[1].R : 0);
    for (int i = blockIdx.x; i < a.NM; i += gridDim.x) {
        float o[3], R[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] = a.poses[(size_t)i * 12 + k];
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = a.poses[(size_t)i * 12 + 3 + k];
        const int map = a.env_map[i / a.M];
        const MapView mv = map_view(a, map, a.prims + a.map_off[map]);
        const int np = mv.count();
        for (int jj = threadIdx.x; jj < Rt; jj += blockDim.x) {
            const int si = jj < R0 ? 0 : 1, j = si ? jj - R0 : jj;
            const Sensor& sen = a.sen[si];
            if (!sen.out || !sen.tape) continue;
            const size_t at = (size_t)i * sen.R + out_index(sen, j);
            const int id = sen.tape[at];
            float v = sen.range;
            if (id == -2) {
                v = 0.f;
            } else if (id >= 0 && id < np) {
                float d[3];
                const float4 db = ray_dir(sen, R, j, d);
                const float t = hit_distance<EXTRA>(mv, id, o, d[0], d[1], d[2]);
                v = fminf(sen.kind == 0 ? t * db.w : t, sen.range);
            }
            sen.out[at] = v;
        }
    }
}

cudaError_t launch_render_hits(const Args& a, int grid, cudaStream_t st) {
    if (a.nc_max > 0 || a.ng_max > 0) k_render_hits<true><<<grid, 256, 0, st>>>(a);
    else k_render_hits<false><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------- render adjoint
// The ray adjoint works in groups of VL = 8 virtual lanes per (step, agent,
// part) item.  A taped adjoint warp holds four items, one per lane group;
// the re-casting adjoint (which needs the whole warp to cull and cast) one
// item, whose VJPs then run on the first group.  Per item, hit rays are
// queued in increasing slot order, VL slots (a block) at a time (a ballot
// per kind keeps the lane order), spheres from the front of the group's
// queue and the other kinds from the back; the queue is flushed after every
// VQ_FLUSH blocks of a sensor and at the end of each sensor, entry q of a
// kind going to virtual lane q mod VL, so the ray VJPs run on full groups
// without divergence between primitive kinds.  Each virtual lane's partial
// sums follow one fixed order that depends only on the set of hit rays, and
// the VL lanes reduce in a fixed tree: the taped and the re-casting
// adjoints, which find the same hits, agree bit for bit.
struct HitQueue {
    int* slot;      // [VQ_CAP] ray slot in the sensor's table
    float* g;       // [VQ_CAP] output cotangent of the ray
    short* id;      // [VQ_CAP] primitive id
    int ns, nr;     // sphere entries from the front, other kinds from the back
    int nblk;       // blocks pushed since the last flush
};

// Queue `h` (0 .. VQ_PER_WARP - 1) of the warp.
__device__ __forceinline__ HitQueue hit_queue(unsigned char* sm, const Args& a, int warp, int h) {
    HitQueue q;
    unsigned char* base = sm + a.sm.vq + (size_t)warp * VQ_BYTES + (size_t)h * (VQ_CAP * 10);
    q.slot = reinterpret_cast<int*>(base);
    q.g = reinterpret_cast<float*>(q.slot + VQ_CAP);
    q.id = reinterpret_cast<short*>(q.g + VQ_CAP);
    q.ns = q.nr = q.nblk = 0;
    return q;
}

// Push the rays of the VL-slot block held by lane group `src` (its lanes'
// valid: a hit with a non-zero cotangent) into q.  Every lane of the warp
// calls it; the lanes whose q is the pushed queue keep its counters.
__device__ __forceinline__ void hq_push(HitQueue& q, int src, bool valid, int ns, int j, int id, float g) {
    const int lane = threadIdx.x & 31;
    const unsigned gmask = ((1u << VL) - 1u) << (VL * src);
    const unsigned below = (1u << lane) - 1u;
    const bool hs = valid && id < ns, hr = valid && id >= ns;
    const unsigned bs = __ballot_sync(0xffffffffu, hs) & gmask, br = __ballot_sync(0xffffffffu, hr) & gmask;
    if (lane / VL == src && (hs || hr)) {
        const int p = hs ? q.ns + __popc(bs & below) : VQ_CAP - 1 - (q.nr + __popc(br & below));
        q.slot[p] = j;
        q.g[p] = g;
        q.id[p] = (short)id;
    }
    q.ns += __popc(bs);
    q.nr += __popc(br);
    ++q.nblk;
}

// Ray VJPs of every entry of q (all of sensor sen: a flush never spans two
// sensors) on the lanes with `active`, virtual lane lane % VL, accumulated
// into the lane's go / gR; the lanes with `reset` empty their queue.  Every
// lane of the warp calls it.
template <bool EXTRA>
__device__ __forceinline__ void hq_flush(HitQueue& q, bool active, bool reset, const Sensor& sen,
                                         const MapView& mv, const float* o, const float* R, float* go,
                                         float* gR) {
    const int vl = threadIdx.x % VL;
    __syncwarp();
    if (active) {
        // queued ids are in range and their cotangents non-zero: the kind of
        // each part of the queue is known, no dispatch on the id
        for (int k = vl; k < q.ns; k += VL) {
            float d[3];
            const float4 db = ray_dir(sen, R, q.slot[k], d);
            ray_vjp_sphere(mv, q.id[k], o, d, db, sen, q.g[k], go, gR);
        }
        for (int k = vl; k < q.nr; k += VL) {
            const int p = VQ_CAP - 1 - k;
            float d[3];
            const float4 db = ray_dir(sen, R, q.slot[p], d);
            if (EXTRA) ray_vjp<EXTRA>(mv, q.id[p], o, d[0], d[1], d[2], db, sen, q.g[p], go, gR);
            else ray_vjp_box(mv, q.id[p] - mv.ns, o, d, db, sen, q.g[p], go, gR);
        }
    }
    __syncwarp();
    if (reset) q.ns = q.nr = q.nblk = 0;
}

// Sum of 12 per-lane values over each group of VL = 8 lanes in a fixed tree
// (reduce-scatter through shuffles of distance 4, 2, 1 on 16 value slots):
// virtual lane v (lane % 8) receives the group's totals of values 2v and
// 2v + 1 (meaningful below 12).
__device__ __forceinline__ float2 group_sum12(const float* v) {
    const int vl = threadIdx.x % VL;
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = k < 12 ? v[k] : 0.f;
#pragma unroll
    for (int w = 4, h = 8; w >= 1; w >>= 1, h >>= 1) {
        const bool hi = (vl & w) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = hi ? a[k] : a[k + h];
            a[k] = (hi ? a[k + h] : a[k]) + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return make_float2(a[0], a[1]);
}

// Slot range [j0, j1) of part `part` of P in a sensor of R rays: 32-slot
// blocks split evenly among the parts (the same for every launch shape).
__device__ __forceinline__ void part_range(int R, int part, int P, int& j0, int& j1) {
    if (P == 1) {
        j0 = 0;
        j1 = R;
        return;
    }
    const int W32 = (R + 31) / 32;
    j0 = 32 * (part * W32 / P);
    j1 = min(R, 32 * ((part + 1) * W32 / P));
}

// (step, agent, part) items reduce, in a fixed order, to the pose cotangent
// gposes[t][i][part] = (d/d origin [3], d/d R [9]); zero when the step
// terminated (the state was replaced).  TAPE: hit ids from the rollout's
// tape, VQ_PER_WARP items per warp (one per lane group); else re-cast, one
// item per warp.
// ONE: a single sensor, as for k_render.
template <int RPT, bool TAPE, bool EXTRA, bool ONE = false>
__global__ void __launch_bounds__(256, TAPE ? 4 : 3) k_render_vjp(const Args a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_env, s_flag, s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int grp = lane / VL, vl = lane % VL;
    const int M = a.M, S = a.S, NM = a.NM;
    const float4* prim = reinterpret_cast<const float4*>(sm + a.sm.prim);
    constexpr bool recast = !TAPE;
    const LCap cap = cap_of(a);
    WList L;
    if (recast) L = wlist_at(sm + a.sm.wlist + (size_t)warp * a.sm.wstride, cap);
    HitQueue hq = hit_queue(sm, a, warp, TAPE ? grp : 0);
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(sm + a.sm.mbar));
    __syncthreads();
    uint32_t phase = 0;
    const int P = a.parts;
    const int per_env = a.T * M * P;
    const int per_warp = TAPE ? VQ_PER_WARP : 1;         // items per warp
    const int lgM = (M & (M - 1)) == 0 ? __ffs(M) - 1 : -1;  // M a power of two: shifts
    const int tasks = (per_env + per_warp - 1) / per_warp;
    for (;;) {
        if (threadIdx.x == 0) {
            s_env = atomicAdd(a.work, 1);
            s_item = NW;
        }
        __syncthreads();
        const int q = s_env;
        if (q >= a.N) break;
        const int env = a.order ? a.order[q] : q;
        const int map = a.env_map[env];
        const MapView mv = map_view(a, map, prim);
        if (!stage_map(a, sm, map, mv, phase, &s_flag)) return;
        prep_boxes(sm, a, mv.ns, mv.nb);
        const int nprim = mv.count();
        for (int task = warp; task < tasks; task = next_item(&s_item, lane)) {
            const int it = TAPE ? VQ_PER_WARP * task + grp : task;  // this lane's item
            const bool has = it < per_env;
            const int itc = has ? it : per_env - 1;
            const int tm = P == 1 ? itc : div_small(itc, P), part = itc - tm * P;
            const int t = lgM >= 0 ? tm >> lgM : div_small(tm, M), m = tm - t * M;
            const size_t ti = (size_t)t * NM + env * M + m;
            const bool live = has && a.done_rd[(size_t)t * NM + env * M] == 0;
            float go[3] = {0.f, 0.f, 0.f}, gR[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) gR[k] = 0.f;
            if (__any_sync(0xffffffffu, live)) {
                float o[3], R[9];
                load_pose(a.poses + ti * 12, o, R);
                auto sensor = [&](const Sensor& sen) {
                    if (!sen.gout || (TAPE && !sen.tape)) return;
                    const size_t base = ti * sen.R;
                    int j0, j1;
                    part_range(sen.R, part, P, j0, j1);
                    if (!live) j1 = j0;  // a terminated step or no item: no block
                    if (TAPE) {
                        // blocks of VL slots per group, all groups in step, in
                        // rounds of 4 whose hit ids and cotangents are loaded
                        // together; a group past its range pushes nothing.
                        // The queue is flushed after every VQ_FLUSH blocks of
                        // the group's range (4 divides VQ_FLUSH, so at a
                        // round's end) and at the sensor's end, as the
                        // re-casting adjoint flushes.
                        const int nb = (j1 - j0 + VL - 1) / VL;
                        int nb_w = nb;
#pragma unroll
                        for (int w = VL; w < 32; w <<= 1) nb_w = max(nb_w, __shfl_xor_sync(0xffffffffu, nb_w, w));
                        const unsigned hm = ((1u << VL) - 1u) << (VL * grp), bl = ((1u << lane) - 1u) & hm;
                        const int16_t* const tp = sen.tape + base;
                        const float* const gp = sen.gout + base;
                        for (int k0 = 0; k0 < nb_w; k0 += 4) {
                            int idv[4];
                            float gv[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int j = j0 + VL * (k0 + u) + vl;
                                idv[u] = -1;
                                gv[u] = 0.f;
                                if (j < j1) {
                                    const int ray = out_index(sen, j);
                                    idv[u] = tp[ray];
                                    gv[u] = gp[ray];
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (k0 + u >= nb_w) break;  // the same on every lane
                                const int id = idv[u];
                                const bool v = (unsigned)id < (unsigned)nprim && gv[u] != 0.f, sph = id < mv.ns;
                                const unsigned bv = __ballot_sync(0xffffffffu, v);
                                const unsigned bs = __ballot_sync(0xffffffffu, v && sph), br = bv & ~bs;
                                if (v) {
                                    const int p = sph ? hq.ns + __popc(bs & bl) : VQ_CAP - 1 - (hq.nr + __popc(br & bl));
                                    hq.slot[p] = j0 + VL * (k0 + u) + vl;
                                    hq.g[p] = gv[u];
                                    hq.id[p] = (short)id;
                                }
                                hq.ns += __popc(bs & hm);
                                hq.nr += __popc(br & hm);
                            }
                            const bool full = k0 + 4 <= nb && (k0 + 4) % VQ_FLUSH == 0;
                            if (__any_sync(0xffffffffu, full)) hq_flush<EXTRA>(hq, full, full, sen, mv, o, R, go, gR);
                        }
                        hq_flush<EXTRA>(hq, true, true, sen, mv, o, R, go, gR);
                        return;
                    }
                    if (__all_sync(0xffffffffu, j0 >= j1)) return;
                    const int4 meta = warp_build_list<EXTRA, true>(mv, o, R, sen, a.cull, L, cap);
                    const int chb = j0 / (32 * RPT), che = (j1 + 32 * RPT - 1) / (32 * RPT);
                    for (int ch = chb; ch < che; ++ch) {
                        float dx[RPT], dy[RPT], dz[RPT], tb[RPT];
                        int bi[RPT];
                        item_rays<RPT>(sen, R, ch, lane, dx, dy, dz, tb);
#pragma unroll
                        for (int r = 0; r < RPT; ++r) bi[r] = -1;
                        if (meta.z < 0) {
                            if (a.cull > 1 && sen.cone) {
                                const int4 nsub = chunk_slots<EXTRA>(L, meta, cap, sen, a.cull, ch, R);
                                cast_sub<RPT, EXTRA>(L, nsub, cap, dx, dy, dz, tb, bi);
                            } else {
                                cast_list<RPT, EXTRA>(L, meta, cap, dx, dy, dz, tb, bi);
                            }
                        }
                        // each 32-slot row: its VL-slot blocks in order, as
                        // the taped gather pushes them; VJPs on the first group
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            const int jb = ch * 32 * RPT + r * 32, j = jb + lane;
                            if (jb >= j1) break;
                            if (jb < j0) continue;
                            const bool hit = j < j1 && meta.z < 0 && bi[r] >= 0;
                            const int id = hit ? L.id[bi[r]] : -1;
                            const float g = hit ? sen.gout[base + out_index(sen, j)] : 0.f;
                            for (int src = 0; src < VQ_PER_WARP; ++src) {
                                if (jb + VL * src >= j1) break;
                                hq_push(hq, src, hit && g != 0.f, mv.ns, j, id, g);
                                if (hq.nblk == VQ_FLUSH) hq_flush<EXTRA>(hq, grp == 0, true, sen, mv, o, R, go, gR);
                            }
                        }
                    }
                    hq_flush<EXTRA>(hq, grp == 0, true, sen, mv, o, R, go, gR);
                    __syncwarp();
                };
                if (ONE) sensor(a.sen[0]);
                else
                    for (int si = 0; si < S; ++si) sensor(a.sen[si]);
            }
            float v12[12];
#pragma unroll
            for (int k = 0; k < 3; ++k) v12[k] = go[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) v12[3 + k] = gR[k];
            const float2 tot = group_sum12(v12);
            if (has && vl < 6 && (TAPE || grp == 0))
                *reinterpret_cast<float2*>(a.gposes + (ti * P + part) * 12 + 2 * vl) = tot;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------- physics adjoint
// One warp per environment, lane per agent.  Segments are taken last to
// first: the segment's states (after resets, replayed from the recorded done
// flags) are recomputed from its checkpoint into the warp's shared-memory
// slice, then steps are reverted: pose cotangent -> state after the step
// (cut by a reset), reward -> state before reset and action, dynamics ->
// previous state.
template <bool EXT>
__global__ void __launch_bounds__(128, EXT ? 4 : 5) k_physics_bwd(const Args a) {
    extern __shared__ __align__(16) float segm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int M = a.M, D = a.c.D, A = a.c.A, NM = a.NM;
    const int Mp = pow2_ceil(M), E = phys_bwd_envs_per_warp(a.K, M);
    const int grp = lane / Mp, agent = lane - grp * Mp, gbase = grp * Mp;
    // environments in the work order (grouped by map, as in the forward: a
    // warp's groups scan maps of one size when the nearest obstacles are
    // recomputed); checkpoints and tapes are indexed by environment
    const int q0 = (blockIdx.x * (blockDim.x >> 5) + wid) * E;
    if (q0 >= a.N) return;
    const bool live = grp < E && q0 + grp < a.N;
    const int qq = live ? q0 + grp : q0;
    const int env = a.order ? a.order[qq] : qq;  // idle groups read a valid environment, write nothing
    float* seg = segm + ((size_t)wid * E + (grp < E ? grp : 0)) * (a.K + 1) * M * 16;
    const int map = a.env_map[env];
    const MapView mv = map_view(a, map, a.prims + a.map_off[map]);
    const bool on = live && agent < M;
    const int i = env * M + (on ? agent : 0);
    const float drag = a.drag_env ? a.drag_env[env] : a.c.drag;
    const float lam = a.lam_env ? a.lam_env[env] : a.c.lam;
    float g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = (on && a.g_sT && k < D) ? a.g_sT[(size_t)i * D + k] : 0.f;
    const int nseg = (a.T + a.K - 1) / a.K;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int t0 = sg * a.K, t1 = min(a.T, t0 + a.K);
        float s[16];
        load_row(a.ckpt + ((size_t)sg * NM + i) * D, D, on, a.c.model, s);
        int kp = a.ckpt_k ? a.ckpt_k[(size_t)sg * a.N + env] : 0;
        if (on)
#pragma unroll
            for (int k = 0; k < 16; ++k) seg[(0 * M + agent) * 16 + k] = s[k];
        for (int t = t0; t < t1; ++t) {
            const bool dn = a.done_rd[(size_t)t * NM + env * M] != 0;
            float act[4], sp[16];
#pragma unroll
            for (int k = 0; k < 4; ++k) act[k] = (on && k < A) ? a.actions[((size_t)t * NM + i) * A + k] : 0.f;
            if (dn && a.c.P > 0 && a.pool) load_row(a.pool + ((size_t)(kp % a.c.P) * NM + i) * D, D, on, a.c.model, sp);
            else step_agent(a.c, drag, lam, s, act, sp);
            if (dn) ++kp;
#pragma unroll
            for (int k = 0; k < 16; ++k) s[k] = sp[k];
            if (on)
#pragma unroll
                for (int k = 0; k < 16; ++k) seg[((t - t0 + 1) * M + agent) * 16 + k] = s[k];
        }
        __syncwarp();
        for (int t = t1 - 1; t >= t0; --t) {
            const size_t o = (size_t)t * NM + i;
            const bool dn = a.done_rd[(size_t)t * NM + env * M] != 0;
            float s0[16], s1[16], act[4];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                s0[k] = on ? seg[((t - t0) * M + agent) * 16 + k] : 0.f;
                s1[k] = on ? seg[((t - t0 + 1) * M + agent) * 16 + k] : 0.f;
            }
            if (!on && a.c.model == MODEL_RIGID) { s0[3] = 1.f; s1[3] = 1.f; }
            if (!on && a.c.model == MODEL_SIMPLE) { s0[6] = s0[10] = s0[14] = 1.f; s1[6] = s1[10] = s1[14] = 1.f; }
#pragma unroll
            for (int k = 0; k < 4; ++k) act[k] = (on && k < A) ? a.actions[o * A + k] : 0.f;
            if (!dn && a.gposes && on) {
                float gq[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) gq[k] = 0.f;
                for (int pp = 0; pp < a.parts; ++pp)  // ray parts in order
#pragma unroll
                    for (int k = 0; k < 12; ++k) gq[k] += a.gposes[(o * a.parts + pp) * 12 + k];
                pose_vjp(a.c.model, s1, gq, gq + 3, g);
            }
            float gp[16], gs[16], gsx[16], ga[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 16; ++k) { gp[k] = dn ? 0.f : g[k]; gs[k] = 0.f; gsx[k] = 0.f; }
            // reward R_ctrl at the state before reset
            float sp[16];
            step_agent(a.c, drag, lam, s0, act, sp);
            int bid;
            if (a.sdf_tape) bid = on ? a.sdf_tape[o] : -1;
            else {
                float sd;
                if (E > 1) nearest_obstacle_lane(mv, sp, sd, bid);
                else nearest_obstacle(mv, M, sp, sd, bid);
            }
            const float gr = (on && a.g_r) ? a.g_r[o] : 0.f;
            if (on) {
                if (EXT && a.c.task == 1) {
                    // progress w_pos (|p_t - g| - |p_{t+1} - g|) towards the taped gate
                    const float4 g0 = mv.gate(a.gate_tape[o])[0];
                    const float e0[3] = {s0[0] - g0.x, s0[1] - g0.y, s0[2] - g0.z};
                    const float e1[3] = {sp[0] - g0.x, sp[1] - g0.y, sp[2] - g0.z};
                    const float n0 = sqrtf(dot3(e0, e0)), n1 = sqrtf(dot3(e1, e1));
                    const float i0 = n0 > 0.f ? 1.f / n0 : 0.f, i1 = n1 > 0.f ? 1.f / n1 : 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        gsx[k] += gr * a.c.w_pos * e0[k] * i0;
                        gp[k] += -gr * a.c.w_pos * e1[k] * i1;
                    }
                } else {
                    const float* tg = a.targets + 3 * (size_t)i;
                    const float e[3] = {sp[0] - tg[0], sp[1] - tg[1], sp[2] - tg[2]};
                    const float ne = sqrtf(dot3(e, e));
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float dpos = a.c.pos_sq ? 2.f * e[k] : (ne > 0.f ? e[k] / ne : 0.f);
                        gp[k] += -gr * a.c.w_pos * dpos;
                    }
                }
                if (EXT && a.g_imu && !dn) imu_vjp(a.c, drag, s0, act, sp, a.g_imu + o * 6, gsx, gp, ga);
                if (a.c.w_obs != 0.f && bid >= 0) {
                    const float sd = sdf_prim(mv, bid, sp);
                    const float ob = relu(a.c.d_safe - sd);
                    if (ob > 0.f) {
                        float gsd[3];
                        sdf_prim_grad(mv, bid, sp, gsd);
#pragma unroll
                        for (int k = 0; k < 3; ++k) gp[k] += gr * 2.f * a.c.w_obs * ob * gsd[k];
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) ga[k] += -2.f * a.c.w_act * gr * act[k];
            }
            for (int n = 0; n < M; ++n) {
                const float px = __shfl_sync(0xffffffffu, sp[0], gbase + n),
                            py = __shfl_sync(0xffffffffu, sp[1], gbase + n),
                            pz = __shfl_sync(0xffffffffu, sp[2], gbase + n),
                            grn = __shfl_sync(0xffffffffu, gr, gbase + n);
                if (n == agent || !on) continue;
                const float dd[3] = {sp[0] - px, sp[1] - py, sp[2] - pz};
                const float dij = sqrtf(dot3(dd, dd));
                const float sv = relu(a.c.d_agent - dij);
                if (sv > 0.f && dij > 0.f) {
                    const float gsum = (gr + grn) * 2.f * a.c.w_agent * sv / dij;
#pragma unroll
                    for (int k = 0; k < 3; ++k) gp[k] += gsum * dd[k];
                }
            }
            // dynamics
            if (a.c.model == MODEL_RIGID) rb_step_vjp(a.c, s0, act, gp, gs, ga);
            else if (a.c.model == MODEL_PMD) pmd_step_vjp(a.c, act, gp, gs, ga);
            else if (a.c.model == MODEL_SIMPLE) simple_step_vjp(a.c, s0, act, gp, gs, ga);
            else pm_step_vjp(a.c, drag, lam, act, gp, gs, ga);
            if (on)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < A) a.g_a[o * A + k] = ga[k];
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = gs[k] + gsx[k];
        }
        __syncwarp();
    }
    if (on && a.g_s0)
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < D) a.g_s0[(size_t)i * D + k] = g[k];
}

// ------------------------------------------------------------ launchers
constexpr int kPhysWarps = 4;

cudaError_t launch_physics(const Args& a, cudaStream_t st) {
    int Mp = 1;
    while (Mp < a.M) Mp <<= 1;
    const int per_cta = kPhysWarps * (32 / Mp);
    const int blocks = (a.N + per_cta - 1) / per_cta;
    if (a.c.task == 1 || a.imu) k_physics<true><<<blocks, 32 * kPhysWarps, 0, st>>>(a);
    else k_physics<false><<<blocks, 32 * kPhysWarps, 0, st>>>(a);
    return cudaGetLastError();
}

// Warps per CTA of the physics adjoint and its dynamic shared memory.
void physics_bwd_shape(int K, int M, int* warps, size_t* smem) {
    const size_t per = (size_t)phys_bwd_envs_per_warp(K, M) * (K + 1) * M * 16 * sizeof(float);
    int w = kPhysWarps;
    while (w > 1 && (size_t)w * per > 96 * 1024) --w;
    *warps = w;
    *smem = (size_t)w * per;
}

cudaError_t launch_physics_bwd(const Args& a, cudaStream_t st) {
    int w;
    size_t smem;
    physics_bwd_shape(a.K, a.M, &w, &smem);
    const bool ext = a.c.task == 1 || a.g_imu;
    cudaError_t e = cudaFuncSetAttribute(ext ? k_physics_bwd<true> : k_physics_bwd<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per_cta = w * phys_bwd_envs_per_warp(a.K, a.M);
    if (ext) k_physics_bwd<true><<<(a.N + per_cta - 1) / per_cta, 32 * w, smem, st>>>(a);
    else k_physics_bwd<false><<<(a.N + per_cta - 1) / per_cta, 32 * w, smem, st>>>(a);
    return cudaGetLastError();
}

template <class K>
static cudaError_t render_launch(K kernel, bool launch, const Args& a, int grid, int block, size_t smem,
                                 cudaStream_t st, int* occ) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!launch) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kernel, block, smem);
    kernel<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// EXTRA kernels read cylinders and gates; maps of spheres and boxes only use
// the kernels compiled without that code.
template <int RPT, bool EXTRA>
static cudaError_t render_rpt(bool vjp, bool launch, const Args& a, int grid, int block, size_t smem,
                              cudaStream_t st, int* occ) {
    const bool one = a.S == 1;
    if (vjp && (a.sen[0].tape || (a.S > 1 && a.sen[1].tape))) {  // taped hit ids: one kernel for every RPT
        if (one) return render_launch(k_render_vjp<1, true, EXTRA, true>, launch, a, grid, block, smem, st, occ);
        return render_launch(k_render_vjp<1, true, EXTRA>, launch, a, grid, block, smem, st, occ);
    }
    if (vjp) return render_launch(k_render_vjp<RPT, false, EXTRA>, launch, a, grid, block, smem, st, occ);
    // shared lists for split items: compiled for the cone-culling default of
    // 4 rays per thread only (the other shapes keep one list per item)
    if constexpr (!EXTRA) {  // warp per ray (one list per item)
        if (a.cast_mode == 1) return render_launch(k_render<RPT, false, false, true>, launch, a, grid, block, smem, st, occ);
    }
    if constexpr (RPT == 4) {
        const bool coop = a.rparts[0] + (a.S > 1 ? a.rparts[1] : 0) > a.S && a.T * a.M * a.S <= block / 32;
        if (coop && launch) return render_launch(k_render<RPT, EXTRA, true>, launch, a, grid, block, smem, st, occ);
    }
    if (one) return render_launch(k_render<RPT, EXTRA, false, false, true>, launch, a, grid, block, smem, st, occ);
    return render_launch(k_render<RPT, EXTRA, false>, launch, a, grid, block, smem, st, occ);
}

template <bool EXTRA>
static cudaError_t render_sel(bool vjp, bool launch, int rpt, const Args& a, int grid, int block, size_t smem,
                              cudaStream_t st, int* occ) {
    switch (rpt) {
        case 1: return render_rpt<1, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 2: return render_rpt<2, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 3: return render_rpt<3, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 4: return render_rpt<4, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 5: return render_rpt<5, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 6: return render_rpt<6, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        case 8: return render_rpt<8, EXTRA>(vjp, launch, a, grid, block, smem, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t render_call(bool vjp, bool launch, int rpt, const Args& a, int grid, int block, size_t smem,
                        cudaStream_t st, int* occ) {
    if (a.nc_max > 0 || a.ng_max > 0) return render_sel<true>(vjp, launch, rpt, a, grid, block, smem, st, occ);
    return render_sel<false>(vjp, launch, rpt, a, grid, block, smem, st, occ);
}

}  // namespace ds
