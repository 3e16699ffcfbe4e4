// sim_kernels.cu -- the persistent fused rollout kernel (dynamics, collision,
// rewards, reset, FOV culling and ray casting for T steps) and its adjoint
// (segment recomputation from checkpoints, reverse sweep of Eq. 5).
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

#include "sim_kernels.cuh"

namespace ds {

__device__ __forceinline__ float4 ld4(const float4* p) { return *p; }

// --------------------------------------------------------------- phase B
// Cull the map for every (agent, sensor) list; record origin-relative data
// in index order (ties resolve to the lowest id), and the lowest id of a
// primitive containing the origin (-1 if none).
__device__ void build_lists(const Args& a, unsigned char* sm, int ns, int nb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int L = a.M * a.S;
    const float4* prim = reinterpret_cast<const float4*>(sm + a.sm.prim);
    const float* pose = reinterpret_cast<const float*>(sm + a.sm.pose);
    for (int Lx = warp; Lx < L; Lx += NW) {
        const int m = Lx / a.S;
        const Sensor& sen = a.sen[Lx % a.S];
        const float* o = pose + m * 12;
        const float* R = o + 3;
        float4* lsph = reinterpret_cast<float4*>(sm + a.sm.lsph) + (size_t)Lx * a.ns_max;
        float* lr2 = reinterpret_cast<float*>(sm + a.sm.lr2) + (size_t)Lx * a.ns_max;
        float4* lbox = reinterpret_cast<float4*>(sm + a.sm.lbox) + (size_t)Lx * a.nb_max * 2;
        short* lid = reinterpret_cast<short*>(sm + a.sm.lid) + (size_t)Lx * (a.ns_max + a.nb_max);
        int4* meta = reinterpret_cast<int4*>(sm + a.sm.lmeta) + Lx;
        int inside = INT_MAX, cnt = 0;
        for (int base = 0; base < ns; base += 32) {
            const int k = base + lane;
            bool keep = false;
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
            float r2 = 0.f;
            if (k < ns) {
                float4 sp = prim[k];
                float oc[3] = {sp.x - o[0], sp.y - o[1], sp.z - o[2]};
                r2 = sp.w * sp.w;
                float C = dot3(oc, oc) - r2;
                if (C <= 0.f) inside = min(inside, k);
                keep = !a.cull || cull_keep(sen, R, oc, sp.w);
                e = make_float4(oc[0], oc[1], oc[2], C);
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                lsph[pos] = e;
                lr2[pos] = r2;
                lid[pos] = (short)k;
            }
            cnt += __popc(bal);
        }
        const int nsk = cnt;
        cnt = 0;
        for (int base = 0; base < nb; base += 32) {
            const int k = base + lane;
            bool keep = false;
            float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
            if (k < nb) {
                float4 bl = prim[ns + 2 * k], bh = prim[ns + 2 * k + 1];
                lo = make_float4(bl.x - o[0], bl.y - o[1], bl.z - o[2], 0.f);
                hi = make_float4(bh.x - o[0], bh.y - o[1], bh.z - o[2], 0.f);
                if (lo.x <= 0.f && hi.x >= 0.f && lo.y <= 0.f && hi.y >= 0.f && lo.z <= 0.f && hi.z >= 0.f)
                    inside = min(inside, ns + k);
                float c[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
                float h[3] = {0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z)};
                keep = !a.cull || cull_keep(sen, R, c, sqrtf(dot3(h, h)));
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int pos = cnt + __popc(bal & ((1u << lane) - 1u));
                lbox[2 * pos] = lo;
                lbox[2 * pos + 1] = hi;
                lid[a.ns_max + pos] = (short)(ns + k);
            }
            cnt += __popc(bal);
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) inside = min(inside, __shfl_xor_sync(0xffffffffu, inside, o2));
        if (lane == 0) *meta = make_int4(nsk, cnt, inside == INT_MAX ? -1 : inside, 0);
    }
}

// --------------------------------------------------------------- phase C
// Cast RPT rays per lane of one work item against its list.  Returns the
// per-ray nearest hit (list slot; spheres 0.., boxes ns_max..) in bi and the
// hit distance in tb.
template <int RPT>
__device__ __forceinline__ void cast_rays(const unsigned char* sm, const Args& a, int Lx, const float* dx,
                                          const float* dy, const float* dz, float* tb, int* bi) {
    const int4 meta = *(reinterpret_cast<const int4*>(sm + a.sm.lmeta) + Lx);
    const float4* lsph = reinterpret_cast<const float4*>(sm + a.sm.lsph) + (size_t)Lx * a.ns_max;
    const float* lr2 = reinterpret_cast<const float*>(sm + a.sm.lr2) + (size_t)Lx * a.ns_max;
    const float4* lbox = reinterpret_cast<const float4*>(sm + a.sm.lbox) + (size_t)Lx * a.nb_max * 2;
    // spheres: the ray misses or cannot beat tb unless disc >= min(tb - b, 0)^2
    // and b >= 0; the root is then refined with the perpendicular-offset form.
    for (int k = 0; k < meta.x; ++k) {
        const float4 e = lsph[k];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            float b = fmaf(dx[r], e.x, fmaf(dy[r], e.y, dz[r] * e.z));
            float disc = fmaf(b, b, -e.w);
            float gg = fminf(tb[r] - b, 0.f);
            float h = fmaf(-gg, gg, disc);
            if (fminf(h, b) >= 0.f) {
                float fx = fmaf(-b, dx[r], e.x), fy = fmaf(-b, dy[r], e.y), fz = fmaf(-b, dz[r], e.z);
                float d2 = fmaxf(lr2[k] - fmaf(fx, fx, fmaf(fy, fy, fz * fz)), 0.f);
                float t = e.w / (b + sqrtf(d2));
                if (t < tb[r]) { tb[r] = t; bi[r] = k; }
            }
        }
    }
    if (meta.y > 0) {
        float ix[RPT], iy[RPT], iz[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            ix[r] = 1.f / (fabsf(dx[r]) < 1e-20f ? copysignf(1e-20f, dx[r]) : dx[r]);
            iy[r] = 1.f / (fabsf(dy[r]) < 1e-20f ? copysignf(1e-20f, dy[r]) : dy[r]);
            iz[r] = 1.f / (fabsf(dz[r]) < 1e-20f ? copysignf(1e-20f, dz[r]) : dz[r]);
        }
        for (int k = 0; k < meta.y; ++k) {
            const float4 lo = lbox[2 * k], hi = lbox[2 * k + 1];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                float t1 = lo.x * ix[r], t2 = hi.x * ix[r];
                float t3 = lo.y * iy[r], t4 = hi.y * iy[r];
                float t5 = lo.z * iz[r], t6 = hi.z * iz[r];
                float tn = fmaxf(fmaxf(fminf(t1, t2), fminf(t3, t4)), fminf(t5, t6));
                float tf = fminf(fminf(fmaxf(t1, t2), fmaxf(t3, t4)), fmaxf(t5, t6));
                if (tn <= tf && tn > 0.f && tn < tb[r]) { tb[r] = tn; bi[r] = a.ns_max + k; }
            }
        }
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

// World directions of the lane's rays of an item; tb starts at the clamp
// distance (invalid rays at -1, which no primitive beats).
template <int RPT>
__device__ __forceinline__ void item_rays(const Sensor& sen, const float* R, int chunk, int lane,
                                          float* dx, float* dy, float* dz, float* fac, float* tb) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int ray = chunk * 32 * RPT + r * 32 + lane;
        const bool valid = ray < sen.R;
        float4 db = valid ? __ldg(sen.dir + ray) : make_float4(1.f, 0.f, 0.f, 1.f);
        dx[r] = fmaf(R[0], db.x, fmaf(R[1], db.y, R[2] * db.z));
        dy[r] = fmaf(R[3], db.x, fmaf(R[4], db.y, R[5] * db.z));
        dz[r] = fmaf(R[6], db.x, fmaf(R[7], db.y, R[8] * db.z));
        fac[r] = db.w;
        tb[r] = valid ? (sen.kind == 0 ? sen.range / db.w : sen.range) : -1.f;
    }
}

// ------------------------------------------------------ map staging (TMA)
// Returns false (and flags SIM_STATUS_TIMEOUT) if the bulk copy never landed.
__device__ bool stage_map(const Args& a, unsigned char* sm, int map, int ns, int nb, uint32_t& phase,
                          int* s_flag) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + a.sm.mbar);
    const uint32_t bytes = (uint32_t)(ns + 2 * nb) * 16u;
    if (bytes == 0) return true;
    if (threadIdx.x == 0) {
        bulk_load(sm + a.sm.prim, a.prims + a.map_off[map], bytes, bar);
        bool ok = mbar_wait(bar, phase);
        if (!ok) {
            atomicOr(a.status, 2);
            mbar_wait(bar, phase);  // give the copy in flight a second bounded chance
        }
        *s_flag = ok ? 1 : 0;
    }
    phase ^= 1u;
    __syncthreads();
    return *s_flag != 0;
}

// ------------------------------------------------------- the rollout kernel
template <int RPT>
__global__ void __launch_bounds__(256, 2) k_rollout(const Args a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_env, s_flag;
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
        const int ns = a.map_ns[map], nb = a.map_nb[map];
        for (int i = threadIdx.x; i < M * 16; i += blockDim.x) {
            const int m = i >> 4, k = i & 15;
            st[i] = k < D ? a.state[(size_t)(env * M + m) * D + k] : 0.f;
        }
        if (!stage_map(a, sm, map, ns, nb, phase, &s_flag)) return;
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
                    else pm_step(a.c, drag, lam, s, act, sp);
                    float best = CUDART_INF_F;
                    int bid = -1;
                    for (int k = lane; k < ns + nb; k += 32) {
                        float d = sdf_prim(prim, ns, k, sp);
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
                // A2: collisions and rewards
                for (int m = warp; m < M; m += NW) {
                    if (lane != 0) continue;
                    const int i = env * M + m;
                    const float* p = spre + m * 16;
                    const float sd = aux[m * 8 + 0];
                    bool col = sd < a.c.r_quad;
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
                        float ak = a.actions[((size_t)t * NM + i) * A + k];
                        aa += ak * ak;
                    }
                    float r = -a.c.w_pos * pos - a.c.w_obs * ob * ob - a.c.w_act * aa - a.c.w_agent * pair;
                    const size_t o = (size_t)t * NM + i;
                    if (a.r_ctrl) a.r_ctrl[o] = r;
                    if (a.r_goal) a.r_goal[o] = (int8_t)(col ? -1 : (ne < a.c.success_radius ? 1 : 0));
                    if (a.sdf_tape) a.sdf_tape[o] = (int16_t)reinterpret_cast<int*>(aux)[m * 8 + 1];
                    aux[m * 8 + 2] = col ? 1.f : 0.f;
                }
                __syncthreads();
                // A3: termination, reset from the pool, new pose
                bool dn = false;
                if (a.c.terminate)
                    for (int m = 0; m < M; ++m) dn = dn || aux[m * 8 + 2] != 0.f;
                for (int m = warp; m < M; m += NW) {
                    if (lane != 0) continue;
                    const int i = env * M + m;
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
                    const size_t o = (size_t)t * NM + i;
                    if (a.done) a.done[o] = dn ? 1 : 0;
                    if (a.done_tape) a.done_tape[o] = dn ? 1 : 0;
                }
                if (dn) ++kpool;
                __syncthreads();
            } else {
                for (int m = warp; m < M; m += NW)
                    if (lane == 0) sensor_pose(a.c.model, st + m * 16, pose + m * 12, pose + m * 12 + 3);
                __syncthreads();
            }
            if (a.S == 0) continue;
            // B: cull
            build_lists(a, sm, ns, nb);
            __syncthreads();
            // C: rays
            const int nit = n_items<RPT>(a);
            for (int it = warp; it < nit; it += NW) {
                const Item I = item_of<RPT>(a, it);
                const Sensor& sen = a.sen[I.sidx];
                if (!sen.out && !sen.tape) continue;
                const float* R = pose + I.m * 12 + 3;
                const int4 meta = *(reinterpret_cast<const int4*>(sm + a.sm.lmeta) + I.Lx);
                const short* lid = reinterpret_cast<const short*>(sm + a.sm.lid) + (size_t)I.Lx * (a.ns_max + a.nb_max);
                float dx[RPT], dy[RPT], dz[RPT], fac[RPT], tb[RPT];
                int bi[RPT];
                item_rays<RPT>(sen, R, I.chunk, lane, dx, dy, dz, fac, tb);
#pragma unroll
                for (int r = 0; r < RPT; ++r) bi[r] = -1;
                if (meta.z < 0) cast_rays<RPT>(sm, a, I.Lx, dx, dy, dz, tb, bi);
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
                    else { v = fminf(tb[r] * (sen.kind == 0 ? fac[r] : 1.f), sen.range); id = lid[bi[r]]; }
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

// ------------------------------------------------------------ ray adjoint
// Cotangent of one ray's output w.r.t. the origin (go) and the world
// direction, folded into the rotation cotangent gR += g_d (x) d_B.  Zero for a
// miss, a clamped output or an origin inside the primitive.
__device__ __forceinline__ void ray_vjp(const float4* prim, int ns, int id, const float* o, float dx, float dy,
                                        float dz, const float4& db, const Sensor& sen, float g, float* go,
                                        float* gR) {
    if (id < 0 || g == 0.f) return;
    const float d[3] = {dx, dy, dz};
    float t, n[3];
    if (id < ns) {
        const float4 s = prim[id];
        const float oc[3] = {s.x - o[0], s.y - o[1], s.z - o[2]};
        const float r2 = s.w * s.w;
        const float C = dot3(oc, oc) - r2;
        if (C <= 0.f) return;
        const float b = dot3(d, oc);
        const float f[3] = {fmaf(-b, d[0], oc[0]), fmaf(-b, d[1], oc[1]), fmaf(-b, d[2], oc[2])};
        const float d2 = fmaxf(r2 - dot3(f, f), 0.f);
        t = C / (b + sqrtf(d2));
        const float ir = 1.f / s.w;
#pragma unroll
        for (int k = 0; k < 3; ++k) n[k] = (t * d[k] - oc[k]) * ir;
    } else {
        const int b = id - ns;
        const float4 lo = prim[ns + 2 * b], hi = prim[ns + 2 * b + 1];
        const float l[3] = {lo.x - o[0], lo.y - o[1], lo.z - o[2]};
        const float u[3] = {hi.x - o[0], hi.y - o[1], hi.z - o[2]};
        float tl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float dk = fabsf(d[k]) < 1e-20f ? copysignf(1e-20f, d[k]) : d[k];
            const float iv = 1.f / dk;
            tl[k] = fminf(l[k] * iv, u[k] * iv);
        }
        int ax = 0;
        if (tl[1] > tl[ax]) ax = 1;
        if (tl[2] > tl[ax]) ax = 2;
        t = tl[ax];
        if (!(t > 0.f)) return;
        n[0] = n[1] = n[2] = 0.f;
        n[ax] = d[ax] > 0.f ? -1.f : 1.f;
    }
    const float fac = sen.kind == 0 ? db.w : 1.f;
    if (t * fac >= sen.range) return;
    const float nd = dot3(n, d);
    const float gt = g * fac / nd;
    const float db3[3] = {db.x, db.y, db.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        go[k] -= gt * n[k];
        const float gdk = -gt * t * n[k];
#pragma unroll
        for (int j = 0; j < 3; ++j) gR[3 * k + j] += gdk * db3[j];
    }
}

// ------------------------------------------------------- the adjoint kernel
// Reverse sweep over checkpoint segments.  For each segment the states are
// recomputed from its checkpoint (resets replayed from the recorded done
// flags), then steps are reverted last to first: ray cotangents -> pose ->
// state; reward -> state before reset and action; dynamics -> previous state.
template <int RPT>
__global__ void __launch_bounds__(256, 2) k_adjoint(const Args a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_env, s_flag;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const int M = a.M, D = a.c.D, A = a.c.A, NM = a.NM;
    const float4* prim = reinterpret_cast<const float4*>(sm + a.sm.prim);
    float* spre = reinterpret_cast<float*>(sm + a.sm.spre);
    float* pose = reinterpret_cast<float*>(sm + a.sm.pose);
    float* aux = reinterpret_cast<float*>(sm + a.sm.aux);
    float* gpose = reinterpret_cast<float*>(sm + a.sm.gpose);
    float* gsm = reinterpret_cast<float*>(sm + a.sm.gs);
    float* seg = reinterpret_cast<float*>(sm + a.sm.seg);
    const bool recast = (a.sen[0].tape == nullptr);
    bool any_g = false;
    for (int si = 0; si < a.S; ++si) any_g = any_g || a.sen[si].gout != nullptr;
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
        const int ns = a.map_ns[map], nb = a.map_nb[map];
        for (int i = threadIdx.x; i < M * 16; i += blockDim.x) {
            const int m = i >> 4, k = i & 15;
            gsm[i] = (k < D && a.g_sT) ? a.g_sT[(size_t)(env * M + m) * D + k] : 0.f;
        }
        if (!stage_map(a, sm, map, ns, nb, phase, &s_flag)) return;
        const float drag = a.drag_env ? a.drag_env[env] : a.c.drag;
        const float lam = a.lam_env ? a.lam_env[env] : a.c.lam;
        const int nseg = (a.T + a.K - 1) / a.K;
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int t0 = sg * a.K, t1 = min(a.T, t0 + a.K);
            for (int i = threadIdx.x; i < M * 16; i += blockDim.x) {
                const int m = i >> 4, k = i & 15;
                seg[i] = k < D ? a.ckpt[((size_t)sg * NM + env * M + m) * D + k] : 0.f;
            }
            int kp = a.ckpt_k ? a.ckpt_k[(size_t)sg * a.N + env] : 0;
            __syncthreads();
            // recompute the segment's states s_t0 .. s_t1 (after resets)
            for (int t = t0; t < t1; ++t) {
                const bool dn = a.done_rd[(size_t)t * NM + env * M] != 0;
                for (int m = warp; m < M; m += NW) {
                    if (lane != 0) continue;
                    const int i = env * M + m;
                    float s[16], sp[16], act[4];
                    const float* cur = seg + ((size_t)(t - t0) * M + m) * 16;
                    float* nxt = seg + ((size_t)(t - t0 + 1) * M + m) * 16;
#pragma unroll
                    for (int k = 0; k < 16; ++k) { s[k] = cur[k]; sp[k] = 0.f; }
#pragma unroll
                    for (int k = 0; k < 4; ++k) act[k] = k < A ? a.actions[((size_t)t * NM + i) * A + k] : 0.f;
                    if (dn && a.c.P > 0 && a.pool) {
                        const float* ps = a.pool + ((size_t)(kp % a.c.P) * NM + i) * D;
#pragma unroll
                        for (int k = 0; k < 16; ++k) sp[k] = k < D ? ps[k] : 0.f;
                    } else if (a.c.model == MODEL_RIGID) rb_step(a.c, s, act, sp);
                    else pm_step(a.c, drag, lam, s, act, sp);
#pragma unroll
                    for (int k = 0; k < 16; ++k) nxt[k] = sp[k];
                }
                if (dn) ++kp;
                __syncthreads();
            }
            // reverse sweep
            for (int t = t1 - 1; t >= t0; --t) {
                const bool dn = a.done_rd[(size_t)t * NM + env * M] != 0;
                const float* s1 = seg + (size_t)(t - t0 + 1) * M * 16;
                const float* s0 = seg + (size_t)(t - t0) * M * 16;
                const bool rays = !dn && any_g && a.S > 0;
                if (rays) {
                    for (int m = warp; m < M; m += NW)
                        if (lane == 0) sensor_pose(a.c.model, s1 + m * 16, pose + m * 12, pose + m * 12 + 3);
                    __syncthreads();
                    if (recast) {
                        build_lists(a, sm, ns, nb);
                        __syncthreads();
                    }
                    const int nit = n_items<RPT>(a);
                    for (int it = warp; it < nit; it += NW) {
                        const Item I = item_of<RPT>(a, it);
                        const Sensor& sen = a.sen[I.sidx];
                        if (!sen.gout) {
                            if (lane < 12) gpose[it * 12 + lane] = 0.f;
                            continue;
                        }
                        const float* o = pose + I.m * 12;
                        const float* R = o + 3;
                        float dx[RPT], dy[RPT], dz[RPT], fac[RPT], tb[RPT];
                        int bi[RPT];
                        item_rays<RPT>(sen, R, I.chunk, lane, dx, dy, dz, fac, tb);
                        const size_t base = ((size_t)t * NM + env * M + I.m) * sen.R;
                        int id[RPT];
                        if (recast) {
                            const int4 meta = *(reinterpret_cast<const int4*>(sm + a.sm.lmeta) + I.Lx);
                            const short* lid =
                                reinterpret_cast<const short*>(sm + a.sm.lid) + (size_t)I.Lx * (a.ns_max + a.nb_max);
#pragma unroll
                            for (int r = 0; r < RPT; ++r) bi[r] = -1;
                            if (meta.z < 0) cast_rays<RPT>(sm, a, I.Lx, dx, dy, dz, tb, bi);
#pragma unroll
                            for (int r = 0; r < RPT; ++r) id[r] = (meta.z >= 0 || bi[r] < 0) ? -1 : lid[bi[r]];
                        } else {
#pragma unroll
                            for (int r = 0; r < RPT; ++r) {
                                const int ray = I.chunk * 32 * RPT + r * 32 + lane;
                                id[r] = ray < sen.R ? sen.tape[base + ray] : -1;
                            }
                        }
                        float go[3] = {0.f, 0.f, 0.f}, gR[9];
#pragma unroll
                        for (int k = 0; k < 9; ++k) gR[k] = 0.f;
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            const int ray = I.chunk * 32 * RPT + r * 32 + lane;
                            if (ray >= sen.R) continue;
                            const float g = sen.gout[base + ray];
                            const float4 db = __ldg(sen.dir + ray);
                            ray_vjp(prim, ns, id[r], o, dx[r], dy[r], dz[r], db, sen, g, go, gR);
                        }
#pragma unroll
                        for (int k = 0; k < 3; ++k) go[k] = warp_sum(go[k]);
#pragma unroll
                        for (int k = 0; k < 9; ++k) gR[k] = warp_sum(gR[k]);
                        if (lane == 0) {
#pragma unroll
                            for (int k = 0; k < 3; ++k) gpose[it * 12 + k] = go[k];
#pragma unroll
                            for (int k = 0; k < 9; ++k) gpose[it * 12 + 3 + k] = gR[k];
                        }
                    }
                    __syncthreads();
                }
                // the step's state before reset (positions for the reward terms)
                for (int m = warp; m < M; m += NW) {
                    const int i = env * M + m;
                    float s[16], sp[16], act[4];
#pragma unroll
                    for (int k = 0; k < 16; ++k) { s[k] = s0[m * 16 + k]; sp[k] = 0.f; }
#pragma unroll
                    for (int k = 0; k < 4; ++k) act[k] = k < A ? a.actions[((size_t)t * NM + i) * A + k] : 0.f;
                    if (a.c.model == MODEL_RIGID) rb_step(a.c, s, act, sp);
                    else pm_step(a.c, drag, lam, s, act, sp);
                    int bid;
                    if (a.sdf_tape) {
                        bid = a.sdf_tape[(size_t)t * NM + i];
                    } else {
                        float best = CUDART_INF_F;
                        bid = -1;
                        for (int k = lane; k < ns + nb; k += 32) {
                            float d = sdf_prim(prim, ns, k, sp);
                            if (d < best) { best = d; bid = k; }
                        }
                        warp_argmin(best, bid);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) spre[m * 16 + k] = sp[k];
                        reinterpret_cast<int*>(aux)[m * 8 + 1] = bid;
                        aux[m * 8 + 2] = a.g_r ? a.g_r[(size_t)t * NM + i] : 0.f;
                    }
                }
                __syncthreads();
                for (int m = warp; m < M; m += NW) {
                    if (lane != 0) continue;
                    const int i = env * M + m;
                    float g[16], gp[16], gs[16], act[4], ga[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int k = 0; k < 16; ++k) { g[k] = gsm[m * 16 + k]; gs[k] = 0.f; }
#pragma unroll
                    for (int k = 0; k < 4; ++k) act[k] = k < A ? a.actions[((size_t)t * NM + i) * A + k] : 0.f;
                    if (rays) {
                        // fixed-order sum of the agent's per-item partials (deterministic)
                        const int ipa = n_items<RPT>(a) / M;
                        float gq[12];
#pragma unroll
                        for (int k = 0; k < 12; ++k) gq[k] = 0.f;
                        for (int j = 0; j < ipa; ++j)
#pragma unroll
                            for (int k = 0; k < 12; ++k) gq[k] += gpose[(m * ipa + j) * 12 + k];
                        pose_vjp(a.c.model, s1 + m * 16, gq, gq + 3, g);
                    }
#pragma unroll
                    for (int k = 0; k < 16; ++k) gp[k] = dn ? 0.f : g[k];
                    // reward R_ctrl at the state before reset
                    const float gr = aux[m * 8 + 2];
                    const float* p = spre + m * 16;
                    const float* tg = a.targets + 3 * (size_t)i;
                    float e[3] = {p[0] - tg[0], p[1] - tg[1], p[2] - tg[2]};
                    const float ne = sqrtf(dot3(e, e));
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float dpos = a.c.pos_sq ? 2.f * e[k] : (ne > 0.f ? e[k] / ne : 0.f);
                        gp[k] += -gr * a.c.w_pos * dpos;
                    }
                    const int bid = reinterpret_cast<int*>(aux)[m * 8 + 1];
                    if (a.c.w_obs != 0.f && bid >= 0) {
                        const float sd = sdf_prim(prim, ns, bid, p);
                        const float ob = relu(a.c.d_safe - sd);
                        if (ob > 0.f) {
                            float gsd[3];
                            sdf_prim_grad(prim, ns, bid, p, gsd);
#pragma unroll
                            for (int k = 0; k < 3; ++k) gp[k] += gr * 2.f * a.c.w_obs * ob * gsd[k];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) ga[k] += -2.f * a.c.w_act * gr * act[k];
                    for (int n = 0; n < M; ++n) {
                        if (n == m) continue;
                        const float* pn = spre + n * 16;
                        float dd[3] = {p[0] - pn[0], p[1] - pn[1], p[2] - pn[2]};
                        const float dij = sqrtf(dot3(dd, dd));
                        const float sv = relu(a.c.d_agent - dij);
                        if (sv > 0.f && dij > 0.f) {
                            const float gsum = (gr + aux[n * 8 + 2]) * 2.f * a.c.w_agent * sv / dij;
#pragma unroll
                            for (int k = 0; k < 3; ++k) gp[k] += gsum * dd[k];
                        }
                    }
                    // dynamics
                    float s[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) s[k] = s0[m * 16 + k];
                    if (a.c.model == MODEL_RIGID) rb_step_vjp(a.c, s, act, gp, gs, ga);
                    else pm_step_vjp(a.c, drag, lam, act, gp, gs, ga);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < A) a.g_a[((size_t)t * NM + i) * A + k] = ga[k];
#pragma unroll
                    for (int k = 0; k < 16; ++k) gsm[m * 16 + k] = gs[k];
                }
                __syncthreads();
            }
        }
        if (a.g_s0)
            for (int i = threadIdx.x; i < M * D; i += blockDim.x) {
                const int m = i / D, k = i - m * D;
                a.g_s0[(size_t)(env * M + m) * D + k] = gsm[m * 16 + k];
            }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers
template <int RPT>
static cudaError_t launch_rpt(bool adjoint, const Args& a, int grid, int block, size_t smem, cudaStream_t st) {
    if (adjoint) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adjoint<RPT><<<grid, block, smem, st>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_rollout<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rollout<RPT><<<grid, block, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <int RPT>
static cudaError_t occupancy_rpt(bool adjoint, int block, size_t smem, int* n) {
    if (adjoint) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_adjoint<RPT>, block, smem);
    }
    cudaError_t e = cudaFuncSetAttribute(k_rollout<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_rollout<RPT>, block, smem);
}

bool rpt_supported(int rpt) {
    return rpt == 1 || rpt == 2 || rpt == 3 || rpt == 4 || rpt == 5 || rpt == 6 || rpt == 8;
}

cudaError_t launch_sim(bool adjoint, int rpt, const Args& a, int grid, int block, size_t smem, cudaStream_t st) {
    switch (rpt) {
        case 1: return launch_rpt<1>(adjoint, a, grid, block, smem, st);
        case 2: return launch_rpt<2>(adjoint, a, grid, block, smem, st);
        case 3: return launch_rpt<3>(adjoint, a, grid, block, smem, st);
        case 4: return launch_rpt<4>(adjoint, a, grid, block, smem, st);
        case 5: return launch_rpt<5>(adjoint, a, grid, block, smem, st);
        case 6: return launch_rpt<6>(adjoint, a, grid, block, smem, st);
        case 8: return launch_rpt<8>(adjoint, a, grid, block, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_sim(bool adjoint, int rpt, int block, size_t smem, int* n) {
    switch (rpt) {
        case 1: return occupancy_rpt<1>(adjoint, block, smem, n);
        case 2: return occupancy_rpt<2>(adjoint, block, smem, n);
        case 3: return occupancy_rpt<3>(adjoint, block, smem, n);
        case 4: return occupancy_rpt<4>(adjoint, block, smem, n);
        case 5: return occupancy_rpt<5>(adjoint, block, smem, n);
        case 6: return occupancy_rpt<6>(adjoint, block, smem, n);
        case 8: return occupancy_rpt<8>(adjoint, block, smem, n);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ds
