// pol.cu -- closed-loop policy MLP (include/policy.h): observation packing,
// the two layers forward (layer 1 on the tensor cores through gemm.cu,
// layer 2 per agent on the CUDA cores), the backward pass (head on the CUDA
// cores, the observation cotangent and the layer-1 weight gradient as two
// tensor-core GEMMs), and the C ABI.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gemm.cuh"
#include "policy.h"
#include "umma.cuh"

using um::img_off;

namespace pl {

constexpr int HID = 256, NA = 4, NSF = 16;
constexpr int HEAD = NA * HID + HID + NA;  // per-block partials: dW2, db1, db2
constexpr int HEAD_BLOCK = 256;

__device__ __forceinline__ float bf(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint16_t tobf(float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&h);
}

// Observation feature f of agent m (0 beyond F and for padding rows).
__device__ __forceinline__ float feature(int m, int f, int N, int Rc, int Rl, const float* s, const float* tg,
                                         const float* dep, const float* lid, float cs, float ls) {
    if (m >= N) return 0.f;
    if (f < 3) return __fsub_rn(s[(size_t)m * 13 + f], tg[(size_t)m * 3 + f]);
    if (f < 13) return s[(size_t)m * 13 + f];
    if (f < 16) return s[(size_t)m * 13 + (f - 13)];
    if (f < 16 + Rc) return __fmul_rn(dep[(size_t)m * Rc + (f - 16)], cs);
    if (f < 16 + Rc + Rl) return __fmul_rn(lid[(size_t)m * Rl + (f - 16 - Rc)], ls);
    return 0.f;
}

// Block: a tile of 64 agents x 64 features (one K-block).  Loads are
// coalesced along each agent's observation row (16-feature spans, 16-byte
// vector loads inside the depth and LiDAR blocks); the tile goes to X (rows =
// agents, K = features) directly and, through shared memory, to X^T (rows =
// features, K = agents) as whole 16-byte chunks of 8 agents.
__global__ void __launch_bounds__(256) k_obs_pack(int N, int Np, int Fp, int Rc, int Rl, const float* s,
                                                  const float* tg, const float* dep, const float* lid, float cs,
                                                  float ls, uint8_t* X, uint8_t* XT) {
    __shared__ uint16_t tile[64][72];
    const int m0 = blockIdx.x * 64, f0 = blockIdx.y * 64;
    const int t = threadIdx.x, r = t >> 2, c16 = (t & 3) * 16;
    const int m = m0 + r, f = f0 + c16;
    float v[16];
    const float* src = nullptr;
    float sc = 1.f;
    // vector loads need 16-byte alignment of the row start and of the base
    const bool dv = (Rc & 3) == 0 && ((uintptr_t)dep & 15) == 0;
    const bool lv = (Rl & 3) == 0 && ((uintptr_t)lid & 15) == 0;
    if (dv && m < N && f >= 16 && f + 16 <= 16 + Rc) {
        src = dep + (size_t)m * Rc + (f - 16);
        sc = cs;
    } else if (lv && (Rc & 3) == 0 && m < N && f >= 16 + Rc && f + 16 <= 16 + Rc + Rl) {
        src = lid + (size_t)m * Rl + (f - 16 - Rc);
        sc = ls;
    }
    if (src) {
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(src + i));
            v[i] = __fmul_rn(x.x, sc); v[i + 1] = __fmul_rn(x.y, sc);
            v[i + 2] = __fmul_rn(x.z, sc); v[i + 3] = __fmul_rn(x.w, sc);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = feature(m, f + i, N, Rc, Rl, s, tg, dep, lid, cs, ls);
    }
    uint16_t b[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) b[i] = tobf(v[i]);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4*>(X + img_off(m, f + 8 * h, Np)) =
            make_uint4(b[8 * h] | (uint32_t)b[8 * h + 1] << 16, b[8 * h + 2] | (uint32_t)b[8 * h + 3] << 16,
                       b[8 * h + 4] | (uint32_t)b[8 * h + 5] << 16, b[8 * h + 6] | (uint32_t)b[8 * h + 7] << 16);
#pragma unroll
    for (int i = 0; i < 16; ++i) tile[r][c16 + i] = b[i];
    __syncthreads();
    for (int q = t; q < 512; q += 256) {
        const int fr = q >> 3, a8 = (q & 7) * 8;
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = tile[a8 + 2 * j][fr] | (uint32_t)tile[a8 + 2 * j + 1][fr] << 16;
        *reinterpret_cast<uint4*>(XT + img_off(f0 + fr, m0 + a8, Fp)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Master parameters -> W1 image (rows = hidden units, K = features), its
// transpose (rows = features, K = hidden), bf16 W2.  Images zeroed before.
__global__ void k_pol_pack(int F, int Fp, const float* P, uint8_t* W1, uint8_t* W1T, uint16_t* W2b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw1 = HID * F;
    if (i < nw1) {
        const int o = i / F, f = i - o * F;
        const uint16_t b = tobf(P[i]);
        *reinterpret_cast<uint16_t*>(W1 + img_off(o, f, HID)) = b;
        *reinterpret_cast<uint16_t*>(W1T + img_off(f, o, Fp)) = b;
    } else if (i >= nw1 + HID && i < nw1 + HID + NA * HID) {
        W2b[i - nw1 - HID] = tobf(P[i]);
    }
}

// Layer 2 per agent (one warp): u = W2 h + b2 (lane l takes hidden units
// l, l + 32, ...; fixed butterfly order), a = tanh(u).
__global__ void k_pol_head(int N, const uint16_t* h, const uint16_t* W2b, const float* b2, float* act, float* y) {
    const int lane = threadIdx.x & 31;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= N) return;
    float acc[NA] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = lane + 32 * j;
        const float hv = bf(h[(size_t)m * HID + k]);
#pragma unroll
        for (int o = 0; o < NA; ++o) acc[o] = fmaf(bf(W2b[o * HID + k]), hv, acc[o]);
    }
#pragma unroll
    for (int o = 0; o < NA; ++o)
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) acc[o] += __shfl_xor_sync(0xffffffffu, acc[o], w);
    if (lane == 0) {
#pragma unroll
        for (int o = 0; o < NA; ++o) {
            const float a = tanhf(acc[o] + b2[o]);
            act[(size_t)m * NA + o] = a;
            y[(size_t)m * NA + o] = a;
        }
    }
}

// Backward of the head and of the SiLU, grid-stride warps over agents
// (rows m < Np; padding rows write zeros): g_u = g_a (1 - a^2), dh = W2^T g_u,
// dz1 = dh silu'(z1) -> bf16 into dZ1 (rows agents, K hidden) and dZ1^T (rows
// hidden, K agents); per-lane partial sums of dW2 = g_u h^T, db1 = sum dz1,
// db2 = sum g_u, combined per block in warp order into part[block][HEAD].
__global__ void __launch_bounds__(HEAD_BLOCK) k_pol_head_bwd(int N, int Np, const float* g_act, const float* y,
                                                             const uint16_t* h, const float* z1,
                                                             const uint16_t* W2b, uint8_t* dZ1, uint8_t* dZ1T,
                                                             float* part) {
    __shared__ float sh[HEAD_BLOCK / 32][HEAD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    float pw[NA][8], pb1[8], pb2[NA];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        pb1[j] = 0.f;
#pragma unroll
        for (int o = 0; o < NA; ++o) pw[o][j] = 0.f;
    }
#pragma unroll
    for (int o = 0; o < NA; ++o) pb2[o] = 0.f;
    for (int m = gw; m < Np; m += nw) {
        if (m >= N) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = lane + 32 * j;
                *reinterpret_cast<uint16_t*>(dZ1 + img_off(m, k, Np)) = 0;
                *reinterpret_cast<uint16_t*>(dZ1T + img_off(k, m, HID)) = 0;
            }
            continue;
        }
        float gu[NA];
#pragma unroll
        for (int o = 0; o < NA; ++o) {
            const float a = y[(size_t)m * NA + o];
            gu[o] = g_act[(size_t)m * NA + o] * (1.f - a * a);
            if (lane == 0) pb2[o] += gu[o];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = lane + 32 * j;
            const float hv = bf(h[(size_t)m * HID + k]);
            float dh = 0.f;
#pragma unroll
            for (int o = 0; o < NA; ++o) {
                dh = fmaf(gu[o], bf(W2b[o * HID + k]), dh);
                pw[o][j] = fmaf(gu[o], hv, pw[o][j]);
            }
            const float z = z1[(size_t)m * HID + k];
            const float sg = __fdividef(1.f, 1.f + __expf(-z));
            const float dz = dh * (sg * (1.f + z * (1.f - sg)));
            pb1[j] += dz;
            const uint16_t b = tobf(dz);
            *reinterpret_cast<uint16_t*>(dZ1 + img_off(m, k, Np)) = b;
            *reinterpret_cast<uint16_t*>(dZ1T + img_off(k, m, HID)) = b;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int k = lane + 32 * j;
#pragma unroll
        for (int o = 0; o < NA; ++o) sh[warp][o * HID + k] = pw[o][j];
        sh[warp][NA * HID + k] = pb1[j];
    }
    if (lane == 0)
#pragma unroll
        for (int o = 0; o < NA; ++o) sh[warp][NA * HID + HID + o] = pb2[o];
    __syncthreads();
    for (int i = threadIdx.x; i < HEAD; i += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < HEAD_BLOCK / 32; ++w) s += sh[w][i];
        part[(size_t)blockIdx.x * HEAD + i] = s;
    }
}

// State part of the observation cotangent: p gets features 0..2 and 13..15,
// q, v, omega features 3..12; added to g_state.
__global__ void k_state_vjp(int N, const float* gf, float* gs) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    const float* g = gf + (size_t)m * NSF;
    float* o = gs + (size_t)m * 13;
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] += g[k] + g[13 + k];
#pragma unroll
    for (int k = 3; k < 13; ++k) o[k] += g[k];
}

// Gradient accumulation: W1 from the K-split partials (split order), b1, W2,
// b2 from the head partials (block order).
__global__ void k_pol_reduce(int F, int Fp, int splits, const float* wpart, int nblk, const float* hpart,
                             float* grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw1 = HID * F, n = nw1 + HID + NA * HID + NA;
    if (i >= n) return;
    float g = 0.f;
    if (i < nw1) {
        const int o = i / F, f = i - o * F;
        for (int s = 0; s < splits; ++s) g += wpart[((size_t)s * HID + o) * Fp + f];
    } else {
        int slot;
        if (i < nw1 + HID) slot = NA * HID + (i - nw1);             // b1
        else if (i < nw1 + HID + NA * HID) slot = i - nw1 - HID;    // W2
        else slot = NA * HID + HID + (i - nw1 - HID - NA * HID);    // b2
        for (int b = 0; b < nblk; ++b) g += hpart[(size_t)b * HEAD + slot];
    }
    grad[i] += g;
}

}  // namespace pl

// ------------------------------------------------------------------ C ABI
struct pol_handle {
    int N = 0, Np = 0, Rc = 0, Rl = 0, F = 0, Fp = 0, num_sms = 0, splits = 1, head_blocks = 0;
    float cs = 0.f, ls = 0.f;
    bool have_act = false;
    float *d_P = nullptr, *d_grad = nullptr;
    uint8_t *d_W1 = nullptr, *d_W1T = nullptr;
    uint16_t* d_W2b = nullptr;
    uint8_t *d_X = nullptr, *d_XT = nullptr, *d_dZ1 = nullptr, *d_dZ1T = nullptr;
    float *d_z1 = nullptr, *d_y = nullptr, *d_gf = nullptr, *d_wpart = nullptr, *d_hpart = nullptr;
    uint16_t* d_h = nullptr;
    int* d_status = nullptr;
    cudaStream_t last = nullptr;
};

namespace {

int crc(cudaError_t e) {
    if (e == cudaSuccess) return SIM_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
}

#define PCK(x)                 \
    do {                       \
        int r_ = crc(x);       \
        if (r_) return r_;     \
    } while (0)

template <class T>
int palloc(T** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return SIM_OK;
    return crc(cudaMalloc((void**)p, bytes));
}

template <class T>
void pfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

size_t nparams(const pol_handle* h) { return (size_t)pl::HID * h->F + pl::HID + pl::NA * pl::HID + pl::NA; }

}  // namespace

extern "C" {

int pol_destroy(pol_handle* h) {
    if (!h) return SIM_OK;
    cudaDeviceSynchronize();
    pfree(h->d_P); pfree(h->d_grad); pfree(h->d_W1); pfree(h->d_W1T); pfree(h->d_W2b);
    pfree(h->d_X); pfree(h->d_XT); pfree(h->d_dZ1); pfree(h->d_dZ1T);
    pfree(h->d_z1); pfree(h->d_y); pfree(h->d_gf); pfree(h->d_wpart); pfree(h->d_hpart); pfree(h->d_h);
    pfree(h->d_status);
    delete h;
    return SIM_OK;
}

int pol_create(int32_t n_env, int32_t cam_rays, float cam_range, int32_t lidar_rays, float lidar_range,
               pol_handle** out) {
    if (!out) return SIM_ERR_NULL_PTR;
    *out = nullptr;
    if (n_env < 1 || n_env > (1 << 24) || cam_rays < 0 || lidar_rays < 0 || cam_rays + lidar_rays > (1 << 20))
        return SIM_ERR_SIZE;
    if ((cam_rays > 0 && !(std::isfinite(cam_range) && cam_range > 0.f)) ||
        (lidar_rays > 0 && !(std::isfinite(lidar_range) && lidar_range > 0.f)))
        return SIM_ERR_INVALID_ARG;
    pol_handle* h = new (std::nothrow) pol_handle();
    if (!h) return SIM_ERR_OOM;
    h->N = n_env;
    h->Np = (n_env + 127) / 128 * 128;
    h->Rc = cam_rays;
    h->Rl = lidar_rays;
    h->F = pl::NSF + cam_rays + lidar_rays;
    h->Fp = (h->F + 63) / 64 * 64;
    h->cs = cam_rays ? 1.f / cam_range : 0.f;
    h->ls = lidar_rays ? 1.f / lidar_range : 0.f;
#define TRY(x)               \
    do {                     \
        int r_ = (x);        \
        if (r_) {            \
            pol_destroy(h);  \
            return r_;       \
        }                    \
    } while (0)
    int dev = 0;
    TRY(crc(cudaGetDevice(&dev)));
    TRY(crc(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev)));
    const size_t Np = h->Np, Fp = h->Fp, np = nparams(h);
    // K splits of the weight-gradient GEMM: about one CTA per SM
    const int tiles = 2 * ((h->Fp + 255) / 256);
    h->splits = std::max(1, std::min((int)(Np / 64), h->num_sms / tiles));
    h->head_blocks = 4 * h->num_sms;
    TRY(palloc(&h->d_P, np * 4)); TRY(palloc(&h->d_grad, np * 4));
    TRY(palloc(&h->d_W1, (size_t)pl::HID * Fp * 2)); TRY(palloc(&h->d_W1T, Fp * pl::HID * 2));
    TRY(palloc(&h->d_W2b, (size_t)pl::NA * pl::HID * 2));
    TRY(palloc(&h->d_X, Np * Fp * 2)); TRY(palloc(&h->d_XT, Fp * Np * 2));
    TRY(palloc(&h->d_dZ1, Np * pl::HID * 2)); TRY(palloc(&h->d_dZ1T, (size_t)pl::HID * Np * 2));
    TRY(palloc(&h->d_z1, Np * pl::HID * 4)); TRY(palloc(&h->d_h, Np * pl::HID * 2));
    TRY(palloc(&h->d_y, (size_t)h->N * pl::NA * 4)); TRY(palloc(&h->d_gf, Np * pl::NSF * 4));
    TRY(palloc(&h->d_wpart, (size_t)h->splits * pl::HID * Fp * 4));
    TRY(palloc(&h->d_hpart, (size_t)h->head_blocks * pl::HEAD * 4));
    TRY(palloc(&h->d_status, 4));
    TRY(crc(cudaMemset(h->d_status, 0, 4)));
    TRY(crc(cudaMemset(h->d_grad, 0, np * 4)));
    std::vector<float> zero(np, 0.f);
    *out = h;
    int rc = pol_set_params(h, zero.data());
    if (rc) {
        *out = nullptr;
        pol_destroy(h);
        return rc;
    }
#undef TRY
    return SIM_OK;
}

int pol_nparams(const pol_handle* h, int64_t* n) {
    if (!h || !n) return SIM_ERR_NULL_PTR;
    *n = (int64_t)nparams(h);
    return SIM_OK;
}

int pol_set_params(pol_handle* h, const float* params) {
    if (!h || !params) return SIM_ERR_NULL_PTR;
    const size_t np = nparams(h);
    for (size_t i = 0; i < np; ++i)
        if (!std::isfinite(params[i])) return SIM_ERR_INVALID_ARG;
    PCK(cudaDeviceSynchronize());
    PCK(cudaMemcpy(h->d_P, params, np * 4, cudaMemcpyHostToDevice));
    PCK(cudaMemset(h->d_W1, 0, (size_t)pl::HID * h->Fp * 2));
    PCK(cudaMemset(h->d_W1T, 0, (size_t)h->Fp * pl::HID * 2));
    pl::k_pol_pack<<<(unsigned)((np + 255) / 256), 256>>>(h->F, h->Fp, h->d_P, h->d_W1, h->d_W1T, h->d_W2b);
    PCK(cudaGetLastError());
    PCK(cudaDeviceSynchronize());
    h->have_act = false;
    return SIM_OK;
}

int pol_get_params(pol_handle* h, float* params) {
    if (!h || !params) return SIM_ERR_NULL_PTR;
    PCK(cudaDeviceSynchronize());
    PCK(cudaMemcpy(params, h->d_P, nparams(h) * 4, cudaMemcpyDeviceToHost));
    return SIM_OK;
}

int pol_act(pol_handle* h, const float* state, const float* targets, const float* depth, const float* lidar,
            float* actions, sim_stream_t stream) {
    if (!h || !state || !targets || !actions) return SIM_ERR_NULL_PTR;
    if ((h->Rc && !depth) || (h->Rl && !lidar)) return SIM_ERR_NULL_PTR;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    pl::k_obs_pack<<<dim3((unsigned)(h->Np / 64), (unsigned)(h->Fp / 64)), 256, 0, st>>>(
        h->N, h->Np, h->Fp, h->Rc, h->Rl, state, targets, depth, lidar, h->cs, h->ls, h->d_X, h->d_XT);
    PCK(cudaGetLastError());
    gm::GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = h->d_X; g.RA = h->Np; g.B = h->d_W1; g.RB = pl::HID;
    g.M = h->N; g.N = pl::HID; g.nkb = h->Fp / 64; g.splits = 1;
    g.epi = gm::EPI_POLICY; g.bias = h->d_P + (size_t)pl::HID * h->F;
    g.z_out = h->d_z1; g.h_out = h->d_h; g.status = h->d_status;
    PCK(gm::launch_gemm(g, st));
    const unsigned hb = (unsigned)(((long long)h->N * 32 + 255) / 256);
    pl::k_pol_head<<<hb, 256, 0, st>>>(h->N, h->d_h, h->d_W2b, h->d_P + nparams(h) - pl::NA, actions, h->d_y);
    PCK(cudaGetLastError());
    h->have_act = true;
    return SIM_OK;
}

int pol_backward(pol_handle* h, const float* g_actions, float* g_state, float* g_depth, float* g_lidar,
                 sim_stream_t stream) {
    if (!h || !g_actions || !g_state) return SIM_ERR_NULL_PTR;
    if ((h->Rc && !g_depth) || (h->Rl && !g_lidar)) return SIM_ERR_NULL_PTR;
    if (!h->have_act) return SIM_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    pl::k_pol_head_bwd<<<h->head_blocks, pl::HEAD_BLOCK, 0, st>>>(h->N, h->Np, g_actions, h->d_y, h->d_h, h->d_z1,
                                                                   h->d_W2b, h->d_dZ1, h->d_dZ1T, h->d_hpart);
    PCK(cudaGetLastError());
    gm::GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.status = h->d_status;
    // observation cotangent: dZ1 (rows agents, K hidden) x W1 -> [N][F]
    g.A = h->d_dZ1; g.RA = h->Np; g.B = h->d_W1T; g.RB = h->Fp;
    g.M = h->N; g.N = h->Fp; g.nkb = pl::HID / 64; g.splits = 1;
    g.epi = gm::EPI_OBS_GRAD; g.g_f = h->d_gf; g.g_cam = g_depth; g.g_lid = g_lidar;
    g.Rc = h->Rc; g.Rl = h->Rl; g.cam_scale = h->cs; g.lid_scale = h->ls;
    PCK(gm::launch_gemm(g, st));
    pl::k_state_vjp<<<(h->N + 255) / 256, 256, 0, st>>>(h->N, h->d_gf, g_state);
    PCK(cudaGetLastError());
    // layer-1 weight gradient: dZ1^T (rows hidden, K agents) x X -> [256][F], K split
    memset(&g, 0, sizeof(g));
    g.status = h->d_status;
    g.A = h->d_dZ1T; g.RA = pl::HID; g.B = h->d_XT; g.RB = h->Fp;
    g.M = pl::HID; g.N = h->Fp; g.nkb = h->Np / 64; g.splits = h->splits;
    g.epi = gm::EPI_STORE; g.C = h->d_wpart; g.ldc = h->Fp;
    PCK(gm::launch_gemm(g, st));
    const size_t np = nparams(h);
    pl::k_pol_reduce<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(h->F, h->Fp, h->splits, h->d_wpart,
                                                                   h->head_blocks, h->d_hpart, h->d_grad);
    PCK(cudaGetLastError());
    return SIM_OK;
}

int pol_grads(pol_handle* h, float* grads, int32_t reset) {
    if (!h || !grads) return SIM_ERR_NULL_PTR;
    PCK(cudaDeviceSynchronize());
    PCK(cudaMemcpy(grads, h->d_grad, nparams(h) * 4, cudaMemcpyDeviceToHost));
    if (reset) PCK(cudaMemset(h->d_grad, 0, nparams(h) * 4));
    return SIM_OK;
}

int pol_last_status(pol_handle* h, int32_t* status) {
    if (!h || !status) return SIM_ERR_NULL_PTR;
    PCK(cudaStreamSynchronize(h->last));
    int v = 0;
    PCK(cudaMemcpy(&v, h->d_status, 4, cudaMemcpyDeviceToHost));
    PCK(cudaMemset(h->d_status, 0, 4));
    *status = v;
    return v & 2 ? SIM_ERR_TIMEOUT : SIM_OK;
}

}  // extern "C"
