// sim_raycast.cuh -- ray casting building blocks shared by the rollout
// kernels: a warp-level field-of-view cull into an origin-relative list, the
// per-lane ray sweep over that list, map staging by TMA bulk copy, and the
// vector-Jacobian product of one ray (Sec. III-B; Eq. 5).
#pragma once
#include <climits>

#include "sim_kernels.cuh"

namespace ds {

// One culled list of an (agent, sensor) pair, origin-relative:
//   sph [ns] float4 (oc.xyz, -sqrt(C)) with C = |oc|^2 - r^2 (sqrt(C) is the
//       tangent length: a ray reaches the sphere iff d.oc >= sqrt(C), and
//       then hits it no farther than sqrt(C)),
//   box [nb][2] float4 (centre - o, tangent length of the bounding sphere or
//       -1e30 when the origin is inside it), (half extents, radius of the
//       bounding sphere),
//   cyl [nc][2] float4 (axis centre - o, bounding tangent), (r^2, half
//       height, 0, bounding radius),
//   gat [ng][3] float4 (centre - o, bounding tangent), (cos yaw, sin yaw,
//       half depth, bounding radius), (w, w + b, origin in local normal and
//       lateral coordinates),
//   sx  [ns] float2 (r^2, r),
//   id  [ns + nb + nc + ng] short (map primitive id of each slot; slots of
//       boxes from ns, cylinders from ns + nb, gates from ns + nb + nc, with
//       the capacities as the bases),
//   sub [same] short (slots kept for the current ray chunk),
//   meta int4 (kept spheres, kept boxes, lowest id of a primitive containing
//       the origin or -1, kept cylinders | kept gates << 16).
struct WList {
    float4* sph;
    float2* sx;
    float4* box;
    float4* cyl;
    float4* gat;
    short* id;
    short* sub;
    int4* meta;
};

__host__ __device__ inline size_t wlist_raw(const LCap& c) {
    return (size_t)16 * (c.ns + 2 * c.nb + 2 * c.nc + 3 * c.ng) + 8 * (size_t)c.ns +
           4 * (size_t)(c.ns + c.nb + c.nc + c.ng);
}

// Bytes of one list laid out contiguously (16-byte aligned parts).
__host__ __device__ inline size_t wlist_bytes(const LCap& c) { return ((wlist_raw(c) + 15) & ~size_t(15)) + 16; }

__device__ inline WList wlist_at(unsigned char* p, const LCap& c) {
    WList L;
    L.sph = reinterpret_cast<float4*>(p);
    L.box = L.sph + c.ns;
    L.cyl = L.box + 2 * c.nb;
    L.gat = L.cyl + 2 * c.nc;
    L.sx = reinterpret_cast<float2*>(L.gat + 3 * c.ng);
    L.id = reinterpret_cast<short*>(L.sx + c.ns);
    L.sub = L.id + c.ns + c.nb + c.nc + c.ng;
    L.meta = reinterpret_cast<int4*>(p + ((wlist_raw(c) + 15) & ~size_t(15)));
    return L;
}

// Packed pairs of the lane's rays: sm_100-class FP32 pair instructions
// (FFMA2 / FMUL2, each element rounded as its scalar counterpart, so results
// are bit-identical to scalar code) halve the issue slots of the tests.
template <int RPT>
struct RayPairs {
    static constexpr int NP = (RPT + 1) / 2;
    float2 x[NP], y[NP], z[NP];
    __device__ __forceinline__ RayPairs(const float* dx, const float* dy, const float* dz) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int r = 2 * p;
            x[p] = make_float2(dx[r], r + 1 < RPT ? dx[r + 1] : 0.f);
            y[p] = make_float2(dy[r], r + 1 < RPT ? dy[r + 1] : 0.f);
            z[p] = make_float2(dz[r], r + 1 < RPT ? dz[r + 1] : 0.f);
        }
    }
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float lo_hi(const float2& v, int q) { return q ? v.y : v.x; }

__device__ __forceinline__ float min3f(float x, float y, float z) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(x), "f"(y), "f"(z));
    return r;
}

__device__ __forceinline__ float max3f(float x, float y, float z) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(x), "f"(y), "f"(z));
    return r;
}

// Box relative to an origin, in the centre / half-extent form the slab test uses.
__device__ __forceinline__ void box_rel(const float4& bl, const float4& bh, const float* o, float* c, float* h) {
    c[0] = 0.5f * (bl.x + bh.x) - o[0];
    c[1] = 0.5f * (bl.y + bh.y) - o[1];
    c[2] = 0.5f * (bl.z + bh.z) - o[2];
    h[0] = 0.5f * (bh.x - bl.x);
    h[1] = 0.5f * (bh.y - bl.y);
    h[2] = 0.5f * (bh.z - bl.z);
}

// Reciprocal of a direction component kept away from 0: the hardware
// approximation (one MUFU operation, at most 1 ulp from the exact value;
// |d| >= 1e-20 keeps operand and result normal, so flushing denormals
// changes nothing).
__device__ __forceinline__ float safe_rcp(float d) {
    const float x = fabsf(d) < 1e-20f ? copysignf(1e-20f, d) : d;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Origin-relative list entries of the four kinds (o: sensor origin).  The
// list builder and hit_distance both build them here, so a recorded hit
// reproduces the cast's distance bit for bit.
// Sphere (c, r): (oc, -sqrt(C)) and (r^2, r), C = |oc|^2 - r^2 (<= 0: inside).
__device__ __forceinline__ bool sphere_list_entry(const float4& sp, const float* o, float4& e, float2& x) {
    const float oc[3] = {sp.x - o[0], sp.y - o[1], sp.z - o[2]};
    const float r2 = sp.w * sp.w;
    const float C = dot3(oc, oc) - r2;
    e = make_float4(oc[0], oc[1], oc[2], -sqrt_approx(fmaxf(C, 0.f)));
    x = make_float2(r2, sp.w);
    return C <= 0.f;
}

// Box corners -> (centre, bounding radius), (half extents, 0).
__device__ __forceinline__ void prep_box(const float4& lo, const float4& hi, float4& cb, float4& hb) {
    const float h[3] = {0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z)};
    cb = make_float4(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z), sqrtf(dot3(h, h)));
    hb = make_float4(h[0], h[1], h[2], 0.f);
}

// Cylinder (axis x, y, radius; z range): (centre - o, bounding tangent) and
// (r^2, half height, 0, bounding radius).  Returns whether o is inside.
__device__ __forceinline__ bool cyl_list_entry(const float4& a0, const float4& a1, const float* o, float4& c0,
                                               float4& c1) {
    const float hz = 0.5f * (a1.y - a1.x);
    const float c[3] = {a0.x - o[0], a0.y - o[1], 0.5f * (a1.x + a1.y) - o[2]};
    const float r2 = a0.z * a0.z;
    const bool in = fmaf(c[0], c[0], c[1] * c[1]) <= r2 && a1.x <= o[2] && a1.y >= o[2];
    const float rho = sqrtf(fmaf(hz, hz, r2));
    const float cb = dot3(c, c) - rho * rho;
    c0 = make_float4(c[0], c[1], c[2], cb > 0.f ? sqrtf(cb) : -1e30f);
    c1 = make_float4(r2, hz, 0.f, rho);
    return in;
}

// Gate frame: (centre - o, bounding tangent), (cos, sin, half depth,
// bounding radius), (opening half size, outer half size, -n.c, -l.c).
// Returns whether o is inside one of its bars.
__device__ __forceinline__ bool gate_list_entry(const float4& a0, const float4& a1, const float* o, float4& g0,
                                                float4& g1, float4& g2) {
    const float W = a0.w + a1.z;
    const float c[3] = {a0.x - o[0], a0.y - o[1], a0.z - o[2]};
    const float un = -fmaf(a1.x, c[0], a1.y * c[1]), ul = -fmaf(a1.x, c[1], -a1.y * c[0]), uz = -c[2];
    const bool in = fabsf(un) <= a1.w && fabsf(ul) <= W && fabsf(uz) <= W && !(fabsf(ul) < a0.w && fabsf(uz) < a0.w);
    const float rho = sqrtf(fmaf(a1.w, a1.w, 2.f * W * W));
    const float cb = dot3(c, c) - rho * rho;
    g0 = make_float4(c[0], c[1], c[2], cb > 0.f ? sqrtf(cb) : -1e30f);
    g1 = make_float4(a1.x, a1.y, a1.w, rho);
    g2 = make_float4(a0.w, W, un, ul);
    return in;
}

// Cull the map for the sensor at origin o with rotation R into L, keeping
// index order within each kind (ties resolve to the lowest id).  Executed
// by one full warp; returns the list's meta.  EXTRA: the map kinds include
// cylinders and gates (else only spheres and boxes are read).
template <bool EXTRA, bool PREP>
__device__ inline int4 warp_build_list(const MapView& mv, const float* o, const float* R, const Sensor& sen,
                                       int cull, const WList& L, const LCap& cap) {
    const int lane = threadIdx.x & 31;
    const float4* prim = mv.prim;
    const int ns = mv.ns, nb = mv.nb;
    const CullK ck = cull_consts(sen);
    int inside = INT_MAX, cnt = 0;
    const unsigned below = (1u << lane) - 1u;
    // One pass per kind: every primitive's bounding sphere is tested against
    // the field of view, and the kept ones get their origin-relative entry
    // at their place in index order (ballot compaction).  A primitive that
    // contains the origin is always kept (its bounding sphere contains the
    // origin and so meets every side plane through it), so the inside test
    // runs on kept primitives only.
    for (int base = 0; base < ns; base += 32) {
        const int k = base + lane;
        const float4 sp = prim[min(k, ns - 1)];
        const float oc[3] = {sp.x - o[0], sp.y - o[1], sp.z - o[2]};
        const bool keep = k < ns && (!cull || cull_keep(ck, R, oc, sp.w));
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int j = cnt + __popc(bal & below);
            float4 e;
            float2 x;
            if (sphere_list_entry(sp, o, e, x)) inside = min(inside, k);
            L.sph[j] = e;
            L.sx[j] = x;
            L.id[j] = (short)k;
        }
        cnt += __popc(bal);
    }
    const int nsk = cnt;
    cnt = 0;
    for (int base = 0; base < nb; base += 32) {
        const int k = base + lane, kc = min(k, nb - 1);
        const float4 bl = prim[ns + 2 * kc];
        float c[3], rho;
        if (PREP) {  // staged as (centre, radius), (half extents, 0)
            c[0] = bl.x - o[0]; c[1] = bl.y - o[1]; c[2] = bl.z - o[2];
            rho = bl.w;
        } else {
            float h[3];
            box_rel(bl, prim[ns + 2 * kc + 1], o, c, h);
            rho = sqrtf(dot3(h, h));
        }
        const bool keep = k < nb && (!cull || cull_keep(ck, R, c, rho));
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int j = cnt + __popc(bal & below);
            const float4 bh = prim[ns + 2 * k + 1];
            float h[3];
            if (PREP) {
                h[0] = bh.x; h[1] = bh.y; h[2] = bh.z;
                if (fabsf(c[0]) <= h[0] && fabsf(c[1]) <= h[1] && fabsf(c[2]) <= h[2]) inside = min(inside, ns + k);
            } else {
                if (bl.x <= o[0] && bh.x >= o[0] && bl.y <= o[1] && bh.y >= o[1] && bl.z <= o[2] && bh.z >= o[2])
                    inside = min(inside, ns + k);
                float cc[3];
                box_rel(bl, bh, o, cc, h);
            }
            // the bounding tangent serves only the chunk cones (cull > 1)
            float tw = -1e30f;
            if (cull > 1) {
                const float cb = dot3(c, c) - rho * rho;
                if (cb > 0.f) tw = sqrtf(cb);
            }
            L.box[2 * j] = make_float4(c[0], c[1], c[2], tw);
            L.box[2 * j + 1] = make_float4(h[0], h[1], h[2], rho);
            L.id[cap.ns + j] = (short)(ns + k);
        }
        cnt += __popc(bal);
    }
    const int nbk = cnt;
    int nck = 0, ngk = 0;
    for (int base = 0; EXTRA && base < mv.nc; base += 32) {
        const int k = base + lane;
        bool keep = false;
        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
        if (k < mv.nc) {
            if (cyl_list_entry(mv.cyl(k)[0], mv.cyl(k)[1], o, c0, c1)) inside = min(inside, ns + nb + k);
            const float c[3] = {c0.x, c0.y, c0.z};
            keep = !cull || cull_keep(ck, R, c, c1.w);
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = nck + __popc(bal & ((1u << lane) - 1u));
            L.cyl[2 * pos] = c0;
            L.cyl[2 * pos + 1] = c1;
            L.id[cap.ns + cap.nb + pos] = (short)(ns + nb + k);
        }
        nck += __popc(bal);
    }
    for (int base = 0; EXTRA && base < mv.ng; base += 32) {
        const int k = base + lane;
        bool keep = false;
        float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0;
        if (k < mv.ng) {
            if (gate_list_entry(mv.gate(k)[0], mv.gate(k)[1], o, g0, g1, g2)) inside = min(inside, ns + nb + mv.nc + k);
            const float c[3] = {g0.x, g0.y, g0.z};
            keep = !cull || cull_keep(ck, R, c, g1.w);
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = ngk + __popc(bal & ((1u << lane) - 1u));
            L.gat[3 * pos] = g0;
            L.gat[3 * pos + 1] = g1;
            L.gat[3 * pos + 2] = g2;
            L.id[cap.ns + cap.nb + cap.nc + pos] = (short)(ns + nb + mv.nc + k);
        }
        ngk += __popc(bal);
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) inside = min(inside, __shfl_xor_sync(0xffffffffu, inside, o2));
    const int4 meta = make_int4(nsk, nbk, inside == INT_MAX ? -1 : inside, nck | (ngk << 16));
    if (lane == 0) *L.meta = meta;
    __syncwarp();
    return meta;
}

// Slab test of one box (centre - origin c, half extents h) against one ray
// given by its reciprocal direction: t = c/d -+ h/|d| per axis, entry = max,
// exit = min; a hit in front of the origin nearer than tb replaces the best.
// |1/d| enters as an operand modifier, so no absolute values are kept.
// 0 <= tn < tb is one unsigned comparison of the bit patterns (a negative tn
// has the sign bit set); tn = +0 means the origin is on the box, a case the
// list's inside test has already taken.
__device__ __forceinline__ void box_test(const float4& c, const float4& h, float ix, float iy, float iz, int slot,
                                         float& tb, int& bi) {
    const float mx = c.x * ix, my = c.y * iy, mz = c.z * iz;
    const float tn = max3f(fmaf(-h.x, fabsf(ix), mx), fmaf(-h.y, fabsf(iy), my), fmaf(-h.z, fabsf(iz), mz));
    const float tf = min3f(fmaf(h.x, fabsf(ix), mx), fmaf(h.y, fabsf(iy), my), fmaf(h.z, fabsf(iz), mz));
    // predicated moves: the update costs two issue slots and no branch
    asm("{\n\t.reg .pred p, q;\n\t"
        "setp.le.f32 p, %2, %3;\n\t"
        "setp.lt.and.u32 q, %4, %5, p;\n\t"
        "@q mov.b32 %0, %2;\n\t"
        "@q mov.b32 %1, %6;\n\t}"
        : "+f"(tb), "+r"(bi)
        : "f"(tn), "f"(tf), "r"(__float_as_uint(tn)), "r"(__float_as_uint(tb)), "r"(slot));
}

// Vertical capped cylinder (list entry c0 = axis centre - o and bounding
// tangent, c1 = (r^2, half height, 0, bounding radius)) against one ray
// with horizontal squared length a = dx^2 + dy^2 (ia = 1/a; vt: the ray is
// parallel to the axis), iz = 1/dz.  Side interval: around the closest
// approach tm = (c.d)/a in the horizontal plane, half-width
// sqrt((r^2 - |c - tm d|^2)/a) (offset form, accurate near tangency); cap
// slab as for boxes; entry = max, exit = min.
__device__ __forceinline__ void cyl_test(const float4& c0, const float4& c1, float dx, float dy, float ia,
                                         bool vt, float iz, int slot, float& tb, int& bi) {
    const float tm = fmaf(dx, c0.x, dy * c0.y) * ia;
    const float fx = fmaf(-tm, dx, c0.x), fy = fmaf(-tm, dy, c0.y);
    const float h2 = (c1.x - fmaf(fx, fx, fy * fy)) * ia;
    const float h = sqrtf(fmaxf(h2, 0.f));
    float t0 = h2 >= 0.f ? tm - h : CUDART_INF_F, t1 = tm + h;
    if (vt) {
        const bool in = fmaf(c0.x, c0.x, c0.y * c0.y) <= c1.x;
        t0 = in ? -CUDART_INF_F : CUDART_INF_F;
        t1 = in ? CUDART_INF_F : -CUDART_INF_F;
    }
    const float mz = c0.z * iz;
    const float tn = fmaxf(t0, fmaf(-c1.y, fabsf(iz), mz)), tf = fminf(t1, fmaf(c1.y, fabsf(iz), mz));
    if (tn <= tf && tn > 0.f && tn < tb) { tb = tn; bi = slot; }
}

// Racing gate (list entry g0 = centre - o and bounding tangent, g1 = (cos,
// sin, half depth, bounding radius), g2 = (w, w + b, origin's local normal
// and lateral coordinates)) against one ray, iz = 1/dz.  Outer box slabs in
// local coordinates give [tn, tf]; the open square prism (lateral and up
// slabs of half-width w) gives (pn, pf).  The first solid point is
// max(tn, 0) unless that lies strictly inside the prism, then the prism's
// exit pf if it is still inside the outer box.
__device__ __forceinline__ float gate_t(const float4& g0, const float4& g1, const float4& g2, float dx, float dy,
                                        float iz, int* axis) {
    const float un = fmaf(g1.x, dx, g1.y * dy), ul = fmaf(g1.x, dy, -g1.y * dx);
    const float in_ = safe_rcp(un), il = safe_rcp(ul);
    const float mn = -g2.z * in_, ml = -g2.w * il, mz = g0.z * iz;
    const float an = fabsf(in_), al = fabsf(il), az = fabsf(iz);
    const float en = fmaf(-g1.z, an, mn), el = fmaf(-g2.y, al, ml), ez = fmaf(-g2.y, az, mz);
    const float tn = max3f(en, el, ez);
    const float tf = min3f(fmaf(g1.z, an, mn), fmaf(g2.y, al, ml), fmaf(g2.y, az, mz));
    const float pn = fmaxf(fmaf(-g2.x, al, ml), fmaf(-g2.x, az, mz));
    const float xl = fmaf(g2.x, al, ml), xz = fmaf(g2.x, az, mz);
    const float pf = fminf(xl, xz);
    const float ta = fmaxf(tn, 0.f);
    const bool in_open = pn < pf && ta > pn && ta < pf;
    const bool hit = tn <= tf && tf >= 0.f && (!in_open || pf <= tf);
    if (axis) {
        // outer entry axis: largest entry time, lowest axis on ties; inner
        // wall: the earlier prism exit, lateral on ties
        const int oa = ez > fmaxf(en, el) ? 2 : (el > en ? 1 : 0);
        *axis = in_open ? (xz < xl ? 4 : 3) : oa;
    }
    return hit ? (in_open ? pf : ta) : CUDART_INF_F;
}

__device__ __forceinline__ void gate_test(const float4& g0, const float4& g1, const float4& g2, float dx, float dy,
                                          float iz, int slot, float& tb, int& bi) {
    const float t = gate_t(g0, g1, g2, dx, dy, iz, nullptr);
    if (t > 0.f && t < tb) { tb = t; bi = slot; }
}

// Near root of a sphere entry e (oc, -sqrt(C)), r2 = r^2, for a ray d that
// reaches it (v = d.oc - sqrt(C) >= 0): perpendicular-offset form
// b - sqrt(r^2 - |oc - b d|^2), b = d.oc.
__device__ __forceinline__ float sphere_near_root(const float4& e, float r2, float v, float dx, float dy, float dz) {
    const float b = v - e.w;
    const float fx = fmaf(-b, dx, e.x), fy = fmaf(-b, dy, e.y), fz = fmaf(-b, dz, e.z);
    const float d2 = fmaxf(r2 - fmaf(fx, fx, fmaf(fy, fy, fz * fz)), 0.f);
    return b - sqrt_approx(d2);
}

// One sphere list entry against the lane's rays: the reach test
// d.oc - sqrt(C) >= 0 on ray pairs, then the near root (perpendicular-offset
// form) for the rays that reach it.
template <int RPT>
__device__ __forceinline__ void sphere_entry(const WList& L, int k, const RayPairs<RPT>& P, float* tb, int* bi) {
    const float4 e = L.sph[k];
#pragma unroll
    for (int p = 0; p < RayPairs<RPT>::NP; ++p) {
        const float2 v2 = __ffma2_rn(P.x[p], f2(e.x), __ffma2_rn(P.y[p], f2(e.y), __ffma2_rn(P.z[p], f2(e.z), f2(e.w))));
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int r = 2 * p + q;
            if (r >= RPT) continue;
            const float v = lo_hi(v2, q);
            if (v >= 0.f) {
                const float t = sphere_near_root(e, L.sx[k].x, v, lo_hi(P.x[p], q), lo_hi(P.y[p], q), lo_hi(P.z[p], q));
                if (t < tb[r]) { tb[r] = t; bi[r] = k; }
            }
        }
    }
}

// Reciprocal directions of the lane's rays (from the packed pairs).
template <int RPT>
struct BoxRays {
    float ix[RPT], iy[RPT], iz[RPT];
    __device__ __forceinline__ explicit BoxRays(const RayPairs<RPT>& P) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            ix[r] = safe_rcp(lo_hi(P.x[r / 2], r & 1));
            iy[r] = safe_rcp(lo_hi(P.y[r / 2], r & 1));
            iz[r] = safe_rcp(lo_hi(P.z[r / 2], r & 1));
        }
    }
};

template <int RPT>
__device__ __forceinline__ void box_entry(const float4& c, const float4& h, const BoxRays<RPT>& B, int slot,
                                          float* tb, int* bi) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) box_test(c, h, B.ix[r], B.iy[r], B.iz[r], slot, tb[r], bi[r]);
}

// Sweep of the cylinder and gate sections of a list (ids from the sub-list
// when sub is set).
template <int RPT>
__device__ __forceinline__ void cast_rest(const WList& L, const LCap& cap, int nck, int ngk, bool sub,
                                          const float* dx, const float* dy, const float* dz, float* tb, int* bi) {
    if (nck <= 0 && ngk <= 0) return;
    float iz[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) iz[r] = safe_rcp(dz[r]);
    if (nck > 0) {
        float ia[RPT];
        bool vt[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const float a = fmaf(dx[r], dx[r], dy[r] * dy[r]);
            vt[r] = a < 1e-12f;
            ia[r] = vt[r] ? 0.f : __frcp_rn(a);
        }
        const int base = cap.ns + cap.nb;
        for (int j = 0; j < nck; ++j) {
            const int k = sub ? L.sub[base + j] : j;
            const float4 c0 = L.cyl[2 * k], c1 = L.cyl[2 * k + 1];
#pragma unroll
            for (int r = 0; r < RPT; ++r) cyl_test(c0, c1, dx[r], dy[r], ia[r], vt[r], iz[r], base + k, tb[r], bi[r]);
        }
    }
    const int base = cap.ns + cap.nb + cap.nc;
    for (int j = 0; j < ngk; ++j) {
        const int k = sub ? L.sub[base + j] : j;
        const float4 g0 = L.gat[3 * k], g1 = L.gat[3 * k + 1], g2 = L.gat[3 * k + 2];
#pragma unroll
        for (int r = 0; r < RPT; ++r) gate_test(g0, g1, g2, dx[r], dy[r], iz[r], base + k, tb[r], bi[r]);
    }
}

// Distance along the ray (origin o, world direction d) to primitive id of
// the map mv (the global map block: boxes as corners), with the entry and
// the test the cast applies to that primitive, so that for a hit the cast
// recorded it equals the cast's distance bit for bit.  +inf if the test
// reports no hit.
template <bool EXTRA>
__device__ __forceinline__ float hit_distance(const MapView& mv, int id, const float* o, float dx, float dy,
                                              float dz) {
    float tb = CUDART_INF_F;
    int bi = -1;
    if (id < mv.ns) {
        float4 e;
        float2 x;
        sphere_list_entry(mv.prim[id], o, e, x);
        const float v = fmaf(dx, e.x, fmaf(dy, e.y, fmaf(dz, e.z, e.w)));  // the cast's packed product, per lane
        return v >= 0.f ? sphere_near_root(e, x.x, v, dx, dy, dz) : CUDART_INF_F;
    }
    if (id < mv.ns + mv.nb) {
        float4 cb, hb;
        prep_box(mv.box(id - mv.ns)[0], mv.box(id - mv.ns)[1], cb, hb);
        const float4 c = make_float4(cb.x - o[0], cb.y - o[1], cb.z - o[2], 0.f);
        box_test(c, hb, safe_rcp(dx), safe_rcp(dy), safe_rcp(dz), 0, tb, bi);
        return tb;
    }
    if (!EXTRA) return CUDART_INF_F;
    const float iz = safe_rcp(dz);
    if (id < mv.ns + mv.nb + mv.nc) {
        float4 c0, c1;
        const int k = id - mv.ns - mv.nb;
        cyl_list_entry(mv.cyl(k)[0], mv.cyl(k)[1], o, c0, c1);
        const float a = fmaf(dx, dx, dy * dy);
        const bool vt = a < 1e-12f;
        cyl_test(c0, c1, dx, dy, vt ? 0.f : __frcp_rn(a), vt, iz, 0, tb, bi);
        return tb;
    }
    float4 g0, g1, g2;
    const int k = id - mv.ns - mv.nb - mv.nc;
    gate_list_entry(mv.gate(k)[0], mv.gate(k)[1], o, g0, g1, g2);
    gate_test(g0, g1, g2, dx, dy, iz, 0, tb, bi);
    return tb;
}

// Sweep RPT rays per lane over a list.  tb holds each ray's best distance
// (start: its clamp distance), bi the list slot of the best hit (spheres
// 0.., boxes cap.ns.., cylinders and gates after).  Sphere: one dot product
// decides whether the ray reaches the sphere (d.oc - sqrt(C) >= 0); only
// then is the near root found (perpendicular-offset form) and compared with
// tb.  Box: slab times in centre / half-extent form, t = c/d -+ h/|d|,
// entry = max, exit = min.
template <int RPT, bool EXTRA>
__device__ __forceinline__ void cast_list(const WList& L, const int4& meta, const LCap& cap, const float* dx,
                                          const float* dy, const float* dz, float* tb, int* bi) {
    const RayPairs<RPT> P(dx, dy, dz);
    for (int k = 0; k < meta.x; ++k) sphere_entry<RPT>(L, k, P, tb, bi);
    if (meta.y > 0) {
        const BoxRays<RPT> B(P);
        for (int k = 0; k < meta.y; ++k) box_entry<RPT>(L.box[2 * k], L.box[2 * k + 1], B, cap.ns + k, tb, bi);
    }
    if (EXTRA && meta.w) cast_rest<RPT>(L, cap, meta.w & 0xffff, meta.w >> 16, false, dx, dy, dz, tb, bi);
}

// Warp per ray: the lanes split the (sub-)list and every ray of the chunk is
// cast by the whole warp in turn, each lane testing its share of the
// entries (spheres: slots lane, lane + 32, ...; then boxes) with the same
// tests as cast_list, a warp-level min-reduction of (t, slot) picking the
// nearest hit and, among equal distances, the lowest slot: the result of the
// per-lane sweep in slot order, bit for bit.  The ray's direction and start
// distance come from the lane that holds it, and its best goes back there.
// Spheres and boxes only.
template <int RPT>
__device__ inline void cast_warp_per_ray(const WList& L, const int4& n, const LCap& cap, bool sub, const float* dx,
                                         const float* dy, const float* dz, float* tb, int* bi) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        for (int l = 0; l < 32; ++l) {
            const float rx = __shfl_sync(0xffffffffu, dx[r], l), ry = __shfl_sync(0xffffffffu, dy[r], l);
            const float rz = __shfl_sync(0xffffffffu, dz[r], l), t0 = __shfl_sync(0xffffffffu, tb[r], l);
            float best = t0;
            int slot = -1;
            for (int j = lane; j < n.x; j += 32) {
                const int k = sub ? L.sub[j] : j;
                const float4 e = L.sph[k];
                const float v = fmaf(rx, e.x, fmaf(ry, e.y, fmaf(rz, e.z, e.w)));
                if (v >= 0.f) {
                    const float t = sphere_near_root(e, L.sx[k].x, v, rx, ry, rz);
                    if (t < best) { best = t; slot = k; }
                }
            }
            if (n.y > 0) {
                const float ix = safe_rcp(rx), iy = safe_rcp(ry), iz = safe_rcp(rz);
                for (int j = lane; j < n.y; j += 32) {
                    const int k = sub ? L.sub[cap.ns + j] : j;
                    box_test(L.box[2 * k], L.box[2 * k + 1], ix, iy, iz, cap.ns + k, best, slot);
                }
            }
            warp_argmin(best, slot);
            if (lane == l) {
                tb[r] = best;
                bi[r] = slot;
            }
        }
    }
}

// Second-level cull for one chunk of rays whose body directions lie in the
// cone (axis cone.xyz, cos = cone.w, sin = sn); aw = R axis in the world.  A
// sphere (or the bounding sphere of a box, cylinder or gate) at oc with
// tangent length sC and radius rho meets the cone iff oc.aw >= cos * sC -
// sin * rho (the angle to the axis at most the half-angle plus the sphere's
// angular radius).  That form holds while the two angles add up to at most
// pi, so a chunk whose half-angle exceeds pi/2 (cos < 0) keeps every entry.
// Writes the kept slots in index order to L.sub (per kind from its slot
// base); one full warp.  Returns the kept counts of the four kinds.
__device__ __forceinline__ bool cone_keep_bound(const float4& c, float rho, const float* aw, float cs, float sn) {
    return cs < 0.f || c.w < 0.f ||
           fmaf(c.x, aw[0], fmaf(c.y, aw[1], fmaf(c.z, aw[2], fmaf(-cs, c.w, sn * rho)))) >= 0.f;
}

template <bool EXTRA>
__device__ inline int4 warp_sub_cull(const WList& L, const int4& meta, const LCap& cap, const float* aw, float cs,
                                     float sn) {
    const int lane = threadIdx.x & 31;
    int ns = 0, nb = 0, nc = 0, ng = 0;
    for (int base = 0; base < meta.x; base += 32) {
        const int k = base + lane;
        bool keep = false;
        if (k < meta.x) {
            const float4 e = L.sph[k];
            const float2 x = L.sx[k];
            keep = cs < 0.f || fmaf(e.x, aw[0], fmaf(e.y, aw[1], fmaf(e.z, aw[2], fmaf(cs, e.w, sn * x.y)))) >= 0.f;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) L.sub[ns + __popc(bal & ((1u << lane) - 1u))] = (short)k;
        ns += __popc(bal);
    }
    for (int base = 0; base < meta.y; base += 32) {
        const int k = base + lane;
        bool keep = false;
        if (k < meta.y) keep = cone_keep_bound(L.box[2 * k], L.box[2 * k + 1].w, aw, cs, sn);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) L.sub[cap.ns + nb + __popc(bal & ((1u << lane) - 1u))] = (short)k;
        nb += __popc(bal);
    }
    const int nck = EXTRA ? meta.w & 0xffff : 0, ngk = EXTRA ? meta.w >> 16 : 0;
    for (int base = 0; base < nck; base += 32) {
        const int k = base + lane;
        const bool keep = k < nck && cone_keep_bound(L.cyl[2 * k], L.cyl[2 * k + 1].w, aw, cs, sn);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) L.sub[cap.ns + cap.nb + nc + __popc(bal & ((1u << lane) - 1u))] = (short)k;
        nc += __popc(bal);
    }
    for (int base = 0; base < ngk; base += 32) {
        const int k = base + lane;
        const bool keep = k < ngk && cone_keep_bound(L.gat[3 * k], L.gat[3 * k + 1].w, aw, cs, sn);
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) L.sub[cap.ns + cap.nb + cap.nc + ng + __popc(bal & ((1u << lane) - 1u))] = (short)k;
        ng += __popc(bal);
    }
    __syncwarp();
    return make_int4(ns, nb, nc, ng);
}

// Sweep RPT rays per lane over the chunk's sub-list (same tests and order as
// cast_list, on the kept slots only).
template <int RPT, bool EXTRA>
__device__ __forceinline__ void cast_sub(const WList& L, const int4& n, const LCap& cap, const float* dx,
                                         const float* dy, const float* dz, float* tb, int* bi) {
    const RayPairs<RPT> P(dx, dy, dz);
    for (int j = 0; j < n.x; ++j) sphere_entry<RPT>(L, L.sub[j], P, tb, bi);
    if (n.y > 0) {
        const BoxRays<RPT> B(P);
        for (int j = 0; j < n.y; ++j) {
            const int k = L.sub[cap.ns + j];
            box_entry<RPT>(L.box[2 * k], L.box[2 * k + 1], B, cap.ns + k, tb, bi);
        }
    }
    if (EXTRA) cast_rest<RPT>(L, cap, n.z, n.w, true, dx, dy, dz, tb, bi);
}

// Slots of a chunk: the sub-cull of the chunk's cone (two-level culling,
// cull > 1) or the whole list.  Returns the sub-list counts.
template <bool EXTRA>
__device__ __forceinline__ int4 chunk_slots(const WList& L, const int4& meta, const LCap& cap, const Sensor& sen,
                                            int cull, int ch, const float* R) {
    const int lane = threadIdx.x & 31;
    if (cull > 1 && sen.cone) {
        const float4 cn = __ldg(sen.cone + ch);
        const float sn = __ldg(sen.cone_sin + ch);
        const float aw[3] = {fmaf(R[0], cn.x, fmaf(R[1], cn.y, R[2] * cn.z)),
                             fmaf(R[3], cn.x, fmaf(R[4], cn.y, R[5] * cn.z)),
                             fmaf(R[6], cn.x, fmaf(R[7], cn.y, R[8] * cn.z))};
        return warp_sub_cull<EXTRA>(L, meta, cap, aw, cn.w, sn);
    }
    const int nck = EXTRA ? meta.w & 0xffff : 0, ngk = EXTRA ? meta.w >> 16 : 0;
    for (int k = lane; k < meta.x; k += 32) L.sub[k] = (short)k;
    for (int k = lane; k < meta.y; k += 32) L.sub[cap.ns + k] = (short)k;
    for (int k = lane; k < nck; k += 32) L.sub[cap.ns + cap.nb + k] = (short)k;
    for (int k = lane; k < ngk; k += 32) L.sub[cap.ns + cap.nb + cap.nc + k] = (short)k;
    __syncwarp();
    return make_int4(meta.x, meta.y, nck, ngk);
}

// Output index of table slot j (rays are stored in tile order when pix is set).
__device__ __forceinline__ int out_index(const Sensor& sen, int j) { return sen.pix ? __ldg(sen.pix + j) : j; }

// Quotient n / d of small non-negative integers (n < 2^21, 0 < d < 2^10)
// through single precision: (n + 0.5) / d is at least 0.5 / d away from an
// integer and the approximate float quotient (2 ulp) errs by less than
// n 2^-22 / d, so its truncation is exact; larger n fall back to integer
// division.
__device__ __forceinline__ int div_small(int n, int d) {
    if (n >= (1 << 21) || d >= (1 << 10)) return n / d;
    return (int)__fdividef((float)n + 0.5f, (float)d);
}

// Next work item of the warp from a shared ticket (dynamic balance).
__device__ __forceinline__ int next_item(int* ticket, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(ticket, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

// World directions and start distances (clamp distances) of the lane's RPT
// rays of chunk `chunk`; a slot past the table gets tb = -1 (never hit).
template <int RPT>
__device__ __forceinline__ void item_rays(const Sensor& sen, const float* R, int chunk, int lane,
                                          float* dx, float* dy, float* dz, float* tb) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int ray = chunk * 32 * RPT + r * 32 + lane;  // table slot
        const bool valid = ray < sen.R;
        float4 db = valid ? __ldg(sen.dir + ray) : make_float4(1.f, 0.f, 0.f, 1.f);
        dx[r] = fmaf(R[0], db.x, fmaf(R[1], db.y, R[2] * db.z));
        dy[r] = fmaf(R[3], db.x, fmaf(R[4], db.y, R[5] * db.z));
        dz[r] = fmaf(R[6], db.x, fmaf(R[7], db.y, R[8] * db.z));
        tb[r] = valid ? __ldg(sen.tmax + ray) : -1.f;
    }
}

// Pose (origin, rotation) of a 12-float record: three 16-byte loads (the
// pose arrays are 16-byte aligned and records 48 bytes apart).
__device__ __forceinline__ void load_pose(const float* p, float* o, float* R) {
    const float4* q = reinterpret_cast<const float4*>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    o[0] = a.x; o[1] = a.y; o[2] = a.z;
    R[0] = a.w; R[1] = b.x; R[2] = b.y; R[3] = b.z; R[4] = b.w;
    R[5] = c.x; R[6] = c.y; R[7] = c.z; R[8] = c.w;
}

// World direction of table slot j.
__device__ __forceinline__ float4 ray_dir(const Sensor& sen, const float* R, int j, float* d) {
    const float4 db = __ldg(sen.dir + j);
    d[0] = fmaf(R[0], db.x, fmaf(R[1], db.y, R[2] * db.z));
    d[1] = fmaf(R[3], db.x, fmaf(R[4], db.y, R[5] * db.z));
    d[2] = fmaf(R[6], db.x, fmaf(R[7], db.y, R[8] * db.z));
    return db;
}

// Sum of 12 per-lane values over the warp in a fixed tree order
// (reduce-scatter: 16 shuffles instead of 60).  Returns, on every lane, the
// total of value (lane >> 1) & 15 (meaningful below 12; lanes 2i and 2i+1
// hold the same total).
__device__ __forceinline__ float warp_sum12(const float* v) {
    const int lane = threadIdx.x & 31;
    float a[8];
    const bool h16 = lane & 16;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float lo = v[k], hi = k + 8 < 12 ? v[k + 8] : 0.f;
        const float send = h16 ? lo : hi;
        a[k] = (h16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    const bool h8 = lane & 8;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float send = h8 ? a[k] : a[k + 4];
        a[k] = (h8 ? a[k + 4] : a[k]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    const bool h4 = lane & 4;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float send = h4 ? a[k] : a[k + 2];
        a[k] = (h4 ? a[k + 2] : a[k]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const bool h2 = lane & 2;
    {
        const float send = h2 ? a[0] : a[1];
        a[0] = (h2 ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// ------------------------------------------------------ map staging (TMA)
// Stage the map block into shared memory with one cp.async.bulk (thread 0
// issues and waits, bounded).  Returns false (and flags SIM_STATUS_TIMEOUT)
// if the bulk copy never landed.
__device__ inline bool stage_map(const Args& a, unsigned char* sm, int map, const MapView& mv, uint32_t& phase,
                                 int* s_flag) {
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + a.sm.mbar);
    const uint32_t bytes = (uint32_t)(mv.ns + 2 * (mv.nb + mv.nc + mv.ng)) * 16u;
    if (bytes == 0) return true;
    if (threadIdx.x == 0) {
        bulk_load(sm + a.sm.prim, a.prims + a.map_off[map], bytes, bar);
        bool ok = mbar_wait_first(bar, phase, a.wait_polls);
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

// Rewrite the staged boxes of a map block from (min, 0), (max, 0) to
// (centre, bounding radius), (half extents, 0), the form every list build
// and ray adjoint of the CTA reads; one pass per environment instead of one
// per (step, agent, sensor) item.  All threads; ends with a block barrier.
__device__ inline void prep_boxes(unsigned char* sm, const Args& a, int ns, int nb) {
    float4* prim = reinterpret_cast<float4*>(sm + a.sm.prim);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        float4 cb, hb;
        prep_box(prim[ns + 2 * b], prim[ns + 2 * b + 1], cb, hb);
        prim[ns + 2 * b] = cb;
        prim[ns + 2 * b + 1] = hb;
    }
    __syncthreads();
}

// Counts of the environment's map, with the block at prim (global or staged).
__device__ __forceinline__ MapView map_view(const Args& a, int map, const float4* prim) {
    MapView m;
    m.prim = prim;
    m.ns = a.map_ns[map];
    m.nb = a.map_nb[map];
    m.nc = a.map_nc ? a.map_nc[map] : 0;
    m.ng = a.map_ng ? a.map_ng[map] : 0;
    return m;
}

// ------------------------------------------------------------ ray adjoint
// Cotangent of one ray's output w.r.t. the origin (go) and the world
// direction, folded into the rotation cotangent gR += g_d (x) d_B.  Zero for a
// miss, a clamped output or an origin inside the primitive.  With the hit
// point's outward normal n: dt/do = -n / (n.d), dt/dd = -t n / (n.d).
// Quotients and the box's slab reciprocals by the hardware approximation (a
// few ulp: the gradient's bar is 1e-3 relative; an entry face that a few ulp
// could change is an edge entry, whose gradient is ambiguous anyway).

// The part shared by every kind: hit distance t, outward normal n.
__device__ __forceinline__ void ray_vjp_tail(float t, const float* n, const float* d, const float4& db,
                                             const Sensor& sen, float g, float* go, float* gR) {
    const float fac = sen.kind == 0 ? db.w : 1.f;
    if (t * fac >= sen.range) return;
    const float nd = dot3(n, d);
    const float gt = __fdividef(g * fac, nd);
    const float db3[3] = {db.x, db.y, db.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        go[k] -= gt * n[k];
        const float gdk = -gt * t * n[k];
#pragma unroll
        for (int j = 0; j < 3; ++j) gR[3 * k + j] += gdk * db3[j];
    }
}

// Sphere id of the map (the caller has checked the id and g != 0).
__device__ __forceinline__ void ray_vjp_sphere(const MapView& mv, int id, const float* o, const float* d,
                                               const float4& db, const Sensor& sen, float g, float* go, float* gR) {
    const float4 s = mv.prim[id];
    const float oc[3] = {s.x - o[0], s.y - o[1], s.z - o[2]};
    const float r2 = s.w * s.w;
    const float C = dot3(oc, oc) - r2;
    if (C <= 0.f) return;
    const float b = dot3(d, oc);
    const float f[3] = {fmaf(-b, d[0], oc[0]), fmaf(-b, d[1], oc[1]), fmaf(-b, d[2], oc[2])};
    const float d2 = fmaxf(r2 - dot3(f, f), 0.f);
    const float t = __fdividef(C, b + sqrt_approx(d2));
    const float ir = __fdividef(1.f, s.w);
    float n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = (t * d[k] - oc[k]) * ir;
    ray_vjp_tail(t, n, d, db, sen, g, go, gR);
}

// Box b of the map, staged as (centre, radius), (half extents, 0) (the
// caller has checked the id and g != 0).
__device__ __forceinline__ void ray_vjp_box(const MapView& mv, int b, const float* o, const float* d,
                                            const float4& db, const Sensor& sen, float g, float* go, float* gR) {
    const float4 bc = mv.prim[mv.ns + 2 * b], bh = mv.prim[mv.ns + 2 * b + 1];
    const float c[3] = {bc.x - o[0], bc.y - o[1], bc.z - o[2]}, h[3] = {bh.x, bh.y, bh.z};
    float tl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float iv = __fdividef(1.f, fabsf(d[k]) < 1e-20f ? copysignf(1e-20f, d[k]) : d[k]);
        tl[k] = fmaf(-h[k], fabsf(iv), c[k] * iv);
    }
    // entry axis: the largest entry time, lowest axis on ties (selects, no
    // runtime-indexed arrays)
    const bool x1 = tl[1] > tl[0];
    const float t01 = x1 ? tl[1] : tl[0];
    const bool x2 = tl[2] > t01;
    const float t = x2 ? tl[2] : t01;
    if (!(t > 0.f)) return;
    const int ax = x2 ? 2 : (x1 ? 1 : 0);
    float n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = k == ax ? (d[k] > 0.f ? -1.f : 1.f) : 0.f;
    ray_vjp_tail(t, n, d, db, sen, g, go, gR);
}

// Any kind, by primitive id (spheres, boxes, then cylinders and gates).
template <bool EXTRA>
__device__ __forceinline__ void ray_vjp(const MapView& mv, int id, const float* o, float dx, float dy, float dz,
                                        const float4& db, const Sensor& sen, float g, float* go, float* gR) {
    if (id < 0 || id >= mv.count() || g == 0.f) return;  // miss (or an id foreign to the map)
    const int ns = mv.ns;
    const float d[3] = {dx, dy, dz};
    if (id < ns) {
        ray_vjp_sphere(mv, id, o, d, db, sen, g, go, gR);
        return;
    }
    if (id < ns + mv.nb) {
        ray_vjp_box(mv, id - ns, o, d, db, sen, g, go, gR);
        return;
    }
    if (!EXTRA) return;
    float t, n[3];
    if (id < ns + mv.nb + mv.nc) {
        const float4 a0 = mv.cyl(id - ns - mv.nb)[0], a1 = mv.cyl(id - ns - mv.nb)[1];
        const float hz = 0.5f * (a1.y - a1.x);
        const float4 c0 = make_float4(a0.x - o[0], a0.y - o[1], 0.5f * (a1.x + a1.y) - o[2], 0.f);
        const float4 c1 = make_float4(a0.z * a0.z, hz, 0.f, 0.f);
        const float a = fmaf(dx, dx, dy * dy);
        const bool vt = a < 1e-12f;
        const float ia = vt ? 0.f : __frcp_rn(a), iz = safe_rcp(dz);
        float tb = CUDART_INF_F;
        int bi = -1;
        cyl_test(c0, c1, dx, dy, ia, vt, iz, 0, tb, bi);
        if (bi < 0) return;
        t = tb;
        // side or cap: the side entry is the later one
        const float tm = fmaf(dx, c0.x, dy * c0.y) * ia;
        const float fx = fmaf(-tm, dx, c0.x), fy = fmaf(-tm, dy, c0.y);
        const float t0 = vt ? -CUDART_INF_F : tm - sqrtf(fmaxf((c1.x - fmaf(fx, fx, fy * fy)) * ia, 0.f));
        const float tz0 = fmaf(-hz, fabsf(iz), c0.z * iz);
        if (t0 >= tz0) {
            const float ir = __fdividef(1.f, a0.z);
            n[0] = fmaf(t, dx, -c0.x) * ir; n[1] = fmaf(t, dy, -c0.y) * ir; n[2] = 0.f;
        } else {
            n[0] = 0.f; n[1] = 0.f; n[2] = dz > 0.f ? -1.f : 1.f;
        }
    } else {
        const float4 a0 = mv.gate(id - ns - mv.nb - mv.nc)[0], a1 = mv.gate(id - ns - mv.nb - mv.nc)[1];
        const float c[3] = {a0.x - o[0], a0.y - o[1], a0.z - o[2]};
        const float4 g0 = make_float4(c[0], c[1], c[2], 0.f);
        const float4 g1 = make_float4(a1.x, a1.y, a1.w, 0.f);
        const float4 g2 = make_float4(a0.w, a0.w + a1.z, -fmaf(a1.x, c[0], a1.y * c[1]),
                                      -fmaf(a1.x, c[1], -a1.y * c[0]));
        int ax;
        t = gate_t(g0, g1, g2, dx, dy, safe_rcp(dz), &ax);
        if (!(t > 0.f) || t == CUDART_INF_F) return;
        // local axis k (0 normal, 1 lateral, 2 up; walls 3 lateral, 4 up):
        // outward normal -sign(d_k) e_k, rotated to the world
        const int k = ax < 3 ? ax : ax - 2;
        const float un = fmaf(a1.x, dx, a1.y * dy), ul = fmaf(a1.x, dy, -a1.y * dx);
        const float dk = k == 0 ? un : (k == 1 ? ul : dz);
        const float sg = dk > 0.f ? -1.f : 1.f;
        n[0] = k == 0 ? sg * a1.x : (k == 1 ? -sg * a1.y : 0.f);
        n[1] = k == 0 ? sg * a1.y : (k == 1 ? sg * a1.x : 0.f);
        n[2] = k == 2 ? sg : 0.f;
    }
    ray_vjp_tail(t, n, d, db, sen, g, go, gR);
}

}  // namespace ds
