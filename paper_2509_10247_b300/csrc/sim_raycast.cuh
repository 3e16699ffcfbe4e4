// sim_raycast.cuh -- ray casting building blocks shared by the rollout
// kernels: a warp-level field-of-view cull into an origin-relative list, the
// per-lane ray sweep over that list, map staging by TMA bulk copy, and the
// vector-Jacobian product of one ray (Sec. III-B; Eq. 5).
#pragma once
#include <climits>

#include "sim_kernels.cuh"

namespace ds {

// One culled list of an (agent, sensor) pair, origin-relative:
//   sph [ns_max] float4 (oc.xyz, C = |oc|^2 - r^2), r2 [ns_max] float (r^2),
//   box [nb_max][2] float4 (lo - o, hi - o), id [ns_max + nb_max] short
//   (map primitive id of each slot; boxes from slot ns_max), meta int4
//   (kept spheres, kept boxes, lowest id of a primitive containing the
//   origin or -1, 0).
struct WList {
    float4* sph;
    float* r2;
    float4* box;
    short* id;
    int4* meta;
};

// Bytes of one list laid out contiguously (16-byte aligned parts).
__host__ __device__ inline size_t wlist_bytes(int ns_max, int nb_max) {
    size_t b = (size_t)16 * (ns_max + 2 * nb_max) + 4 * (size_t)ns_max + 2 * (size_t)(ns_max + nb_max);
    return ((b + 15) & ~size_t(15)) + 16;
}

__device__ inline WList wlist_at(unsigned char* p, int ns_max, int nb_max) {
    WList L;
    L.sph = reinterpret_cast<float4*>(p);
    L.box = L.sph + ns_max;
    L.r2 = reinterpret_cast<float*>(L.box + 2 * nb_max);
    L.id = reinterpret_cast<short*>(L.r2 + ns_max);
    size_t b = (size_t)16 * (ns_max + 2 * nb_max) + 4 * (size_t)ns_max + 2 * (size_t)(ns_max + nb_max);
    L.meta = reinterpret_cast<int4*>(p + ((b + 15) & ~size_t(15)));
    return L;
}

// Cull the map (ns spheres then nb boxes at prim) for the sensor at origin o
// with rotation R into L, keeping index order (ties resolve to the lowest
// id).  Executed by one full warp; returns the list's meta.
__device__ inline int4 warp_build_list(const float4* prim, int ns, int nb, const float* o, const float* R,
                                       const Sensor& sen, int cull, const WList& L, int ns_max) {
    const int lane = threadIdx.x & 31;
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
            keep = !cull || cull_keep(sen, R, oc, sp.w);
            e = make_float4(oc[0], oc[1], oc[2], C);
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            L.sph[pos] = e;
            L.r2[pos] = r2;
            L.id[pos] = (short)k;
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
            keep = !cull || cull_keep(sen, R, c, sqrtf(dot3(h, h)));
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = cnt + __popc(bal & ((1u << lane) - 1u));
            L.box[2 * pos] = lo;
            L.box[2 * pos + 1] = hi;
            L.id[ns_max + pos] = (short)(ns + k);
        }
        cnt += __popc(bal);
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) inside = min(inside, __shfl_xor_sync(0xffffffffu, inside, o2));
    const int4 meta = make_int4(nsk, cnt, inside == INT_MAX ? -1 : inside, 0);
    if (lane == 0) *L.meta = meta;
    __syncwarp();
    return meta;
}

// Sweep RPT rays per lane over a list.  tb holds each ray's best distance
// (start: its clamp distance), bi the list slot of the best hit (spheres
// 0.., boxes ns_max..).  Spheres: the ray misses or cannot beat tb unless
// disc >= min(tb - b, 0)^2 and b >= 0, then the root is refined with the
// perpendicular-offset form.  Boxes: slabs with correctly rounded reciprocals.
template <int RPT>
__device__ __forceinline__ void cast_list(const WList& L, const int4& meta, int ns_max, const float* dx,
                                          const float* dy, const float* dz, float* tb, int* bi) {
    for (int k = 0; k < meta.x; ++k) {
        const float4 e = L.sph[k];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            float b = fmaf(dx[r], e.x, fmaf(dy[r], e.y, dz[r] * e.z));
            float disc = fmaf(b, b, -e.w);
            float gg = fminf(tb[r] - b, 0.f);
            float h = fmaf(-gg, gg, disc);
            if (fminf(h, b) >= 0.f) {
                float fx = fmaf(-b, dx[r], e.x), fy = fmaf(-b, dy[r], e.y), fz = fmaf(-b, dz[r], e.z);
                float d2 = fmaxf(L.r2[k] - fmaf(fx, fx, fmaf(fy, fy, fz * fz)), 0.f);
                float t = e.w / (b + sqrtf(d2));
                if (t < tb[r]) { tb[r] = t; bi[r] = k; }
            }
        }
    }
    if (meta.y > 0) {
        float ix[RPT], iy[RPT], iz[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            ix[r] = __frcp_rn(fabsf(dx[r]) < 1e-20f ? copysignf(1e-20f, dx[r]) : dx[r]);
            iy[r] = __frcp_rn(fabsf(dy[r]) < 1e-20f ? copysignf(1e-20f, dy[r]) : dy[r]);
            iz[r] = __frcp_rn(fabsf(dz[r]) < 1e-20f ? copysignf(1e-20f, dz[r]) : dz[r]);
        }
        for (int k = 0; k < meta.y; ++k) {
            const float4 lo = L.box[2 * k], hi = L.box[2 * k + 1];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                float t1 = lo.x * ix[r], t2 = hi.x * ix[r];
                float t3 = lo.y * iy[r], t4 = hi.y * iy[r];
                float t5 = lo.z * iz[r], t6 = hi.z * iz[r];
                float tn = fmaxf(fmaxf(fminf(t1, t2), fminf(t3, t4)), fminf(t5, t6));
                float tf = fminf(fminf(fmaxf(t1, t2), fmaxf(t3, t4)), fmaxf(t5, t6));
                if (tn <= tf && tn > 0.f && tn < tb[r]) { tb[r] = tn; bi[r] = ns_max + k; }
            }
        }
    }
}

// Next work item of the warp from a shared ticket (dynamic balance).
__device__ __forceinline__ int next_item(int* ticket, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(ticket, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

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
        tb[r] = valid ? __ldg(sen.tmax + ray) : -1.f;
    }
}

// ------------------------------------------------------ map staging (TMA)
// Stage the map block into shared memory with one cp.async.bulk (thread 0
// issues and waits, bounded).  Returns false (and flags SIM_STATUS_TIMEOUT) if the bulk copy never landed.
__device__ inline bool stage_map(const Args& a, unsigned char* sm, int map, int ns, int nb, uint32_t& phase,
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
            const float iv = __frcp_rn(dk);
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

}  // namespace ds
