// surr_train.cu -- one Adam step of the surrogate MLP on a minibatch of
// simulator transitions, on the tensor cores.
//
//   k_surr_fwd_train  per 128-row tile: gather, normalise, three MMAs; keeps
//                     the pre-activations z1, z2 (fp32), writes the inputs
//                     and activations transposed (bf16 images [feature][batch])
//                     for the weight gradients, the loss cotangent dY and its
//                     transpose, loss and dY column sums per tile.
//   k_surr_bwd_train  per tile: dH2 = dY W3 (one MMA), dZ2 = dH2 silu'(z2),
//                     dH1 = dZ2 W2 (16 MMAs), dZ1 = dH1 silu'(z1); writes dZ2,
//                     dZ1 transposed and their column sums.
//   k_surr_wgrad      dW = dZ^T X over the batch (K = batch), split-K over
//                     CTAs, 4-stage bulk-copy pipeline, partials per split.
//   k_surr_adam       sums the partials in a fixed order, Adam update of the
//                     fp32 master weights, re-packs the bf16 images.
#include "surr_kernels.cuh"
#include "umma.cuh"

namespace sg {
using namespace um;


constexpr uint32_t SMEM_TR = IMG_A + IMG_W2 + IMG_H;
constexpr uint32_t SMEM_TR_LAUNCH = SMEM_TR + 1024 + 64;
constexpr int WG_STAGES = 4;
constexpr uint32_t WG_STAGE = 16384 + 32768;
constexpr uint32_t SMEM_WG_LAUNCH = WG_STAGES * WG_STAGE + 1024 + 128;

// SiLU and its derivative with the fast exponential and division (a few
// ulp of fp32; activations and cotangents are rounded to bf16 right after).
__device__ __forceinline__ float silu_t(float z) { return __fdividef(z, 1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu_t(float z) {
    const float sg = __fdividef(1.f, 1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}

__device__ __forceinline__ void st_chunk_t(uint8_t* blk, uint32_t r, uint32_t c, uint4 v) {
    *reinterpret_cast<uint4*>(blk + r * 128u + (((c ^ r) & 7u) << 4)) = v;
}

// Element (row f, column b) of a bf16 image with R rows.
__device__ __forceinline__ void st_img(uint8_t* img, uint32_t R, uint32_t f, uint32_t b, float v) {
    *reinterpret_cast<__nv_bfloat16*>(img + img_off(f, b, R)) = __float2bfloat16_rn(v);
}

// Lane l returns the warp total of v[l] (reduce-scatter in a fixed tree order).
__device__ __forceinline__ float warp_rs32(float* v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool hi = lane & w;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = hi ? v[k] : v[k + w];
            const float keep = hi ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

__device__ __forceinline__ bool sync_wait_t(uint64_t* bar, uint32_t& ph) {
    const bool ok = __syncthreads_and(mbar_wait(bar, ph)) != 0;
    ph ^= 1u;
    return ok;
}

// Common prologue of the per-tile kernels: barriers, 512 tensor-memory
// columns, two weight images into shared memory.  Returns false (status
// flagged) if the copies did not land.
__device__ __forceinline__ bool tile_prologue(uint8_t* sm, uint32_t smem_imgs, const uint8_t* g0, uint32_t n0,
                                              const uint8_t* g1, uint32_t n1, uint32_t off1, int* status,
                                              uint32_t& tmem) {
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + smem_imgs);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + smem_imgs + 16);
    int* sflag = reinterpret_cast<int*>(sm + smem_imgs + 20);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        *sflag = 1;
    }
    __syncthreads();
    if ((tid >> 5) == 0) tmem_alloc(tslot, 512);
    if (tid == 0) {
        mbar_expect_tx(&bars[0], n0 + n1);
        bulk_g2s(sm, g0, n0, &bars[0]);
        bulk_g2s(sm + off1, g1, n1, &bars[0]);
        if (!mbar_wait(&bars[0], 0)) {
            atomicOr(status, 2);
            *sflag = 0;
            mbar_wait(&bars[0], 0);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *tslot;
    return *sflag != 0;
}

__device__ __forceinline__ void tile_epilogue(uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------- forward
__global__ void __launch_bounds__(256, 1) k_surr_fwd_train(const TrainArgs a) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    uint8_t* sm = smraw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* imgA = sm;
    uint8_t* imgW2 = sm + IMG_A;
    uint8_t* imgH = sm + IMG_A + IMG_W2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + SMEM_TR);
    float* red = reinterpret_cast<float*>(sm + SMEM_TR + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t q = warp & 3, half = warp >> 2, r = 32u * q + lane;
    uint32_t tmem;
    bool ok = tile_prologue(sm, SMEM_TR, a.imgA, IMG_A, a.imgW2, IMG_W2, IMG_A, a.status, tmem);
    const uint32_t sA = smem_u32(imgA), sW2 = smem_u32(imgW2), sH = smem_u32(imgH);
    const uint32_t tq = tmem + ((32u * q) << 16);
    const float* st = a.stats;
    const int tile = blockIdx.x;
    const uint32_t b = (uint32_t)tile * 128u + r;  // minibatch row
    uint32_t ph = 0;
    float tgt[13];
    if (tid < 128) {
        const int src = a.idx[b];
        float x[17];
#pragma unroll
        for (int k = 0; k < 17; ++k) x[k] = a.X[(size_t)src * 17 + k];
#pragma unroll
        for (int k = 13; k < 17; ++k) x[k] = ds::clip1(x[k]);
#pragma unroll
        for (int k = 0; k < 13; ++k)
            tgt[k] = __fmul_rn(__fsub_rn(__fsub_rn(a.S1[(size_t)src * 13 + k], x[k]), st[ST_MUD + k]), st[ST_RSD + k]);
        float xh[32];
#pragma unroll
        for (int k = 0; k < 17; ++k) xh[k] = __fmul_rn(__fsub_rn(x[k], st[ST_MUX + k]), st[ST_RSX + k]);
#pragma unroll
        for (int k = 17; k < 32; ++k) xh[k] = 0.f;
        uint32_t p[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) p[i] = pack_bf16(xh[2 * i], xh[2 * i + 1]);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            st_chunk_t(imgA, r, 4 + j, make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]));
#pragma unroll
        for (int k = 0; k < 32; ++k) st_img(a.xT, 32, k, b, xh[k]);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (ok && tid == 0) {
        tc_fence_after();
#pragma unroll
        for (uint32_t ks = 0; ks < 2; ++ks)
            mma_bf16(tmem, desc_sw128(sA + 64 + 32 * ks), desc_sw128(sA + 32 * ks), idesc_bf16(128, 256), ks);
        mma_commit(&bars[1]);
    }
    for (int layer = 0; layer < 2 && ok; ++layer) {
        if (!(ok = sync_wait_t(&bars[1], ph))) break;
        tc_fence_after();
        float* zout = layer == 0 ? a.z1 : a.z2;
        uint8_t* hT = layer == 0 ? a.h1T : a.h2T;
        const float* bias = a.bias + 256 * layer;
#pragma unroll 1
        for (uint32_t c = 0; c < 4; ++c) {
            const uint32_t col0 = half * 128 + 32 * c;
            float v[32];
            tmem_ld32(tq + 256 * layer + col0, v);
            uint32_t p[16];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += __ldg(bias + col0 + i);
#pragma unroll
            for (int i = 0; i < 32; i += 4)
                *reinterpret_cast<float4*>(zout + (size_t)b * 256 + col0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
#pragma unroll
            for (int i = 0; i < 16; ++i) p[i] = pack_bf16(silu_t(v[2 * i]), silu_t(v[2 * i + 1]));
            uint8_t* blk = imgH + (col0 >> 6) * 16384u;
            const uint32_t c0 = (col0 & 63u) >> 3;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                st_chunk_t(blk, r, c0 + j, make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]));
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&p[i]);
                *reinterpret_cast<__nv_bfloat16*>(hT + img_off(col0 + 2 * i, b, 256)) = h2.x;
                *reinterpret_cast<__nv_bfloat16*>(hT + img_off(col0 + 2 * i + 1, b, 256)) = h2.y;
            }
        }
        tc_fence_before();
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            if (layer == 0) {
#pragma unroll
                for (uint32_t ks = 0; ks < 16; ++ks) {
                    const uint32_t kb = ks >> 2, off = (ks & 3) * 32;
                    mma_bf16(tmem + 256, desc_sw128(sH + kb * 16384 + off), desc_sw128(sW2 + kb * 32768 + off),
                             idesc_bf16(128, 256), ks);
                }
            } else {
#pragma unroll
                for (uint32_t ks = 0; ks < 16; ++ks) {
                    const uint32_t adr = sH + (ks >> 2) * 16384 + (ks & 3) * 32;
                    const uint32_t bdr = sA + (128 + 16 * (ks >> 1)) * 128 + 64 + (ks & 1) * 32;
                    mma_bf16(tmem, desc_sw128(adr), desc_sw128(bdr), idesc_bf16(128, 16), ks);
                }
            }
            mma_commit(&bars[1]);
        }
    }
    if (ok) ok = sync_wait_t(&bars[1], ph);
    if (ok) {
        tc_fence_after();
        if (tid < 128) {
            float y[16];
            tmem_ld16(tq, y);
            const float sc = 2.f / (float)(a.B * NOUT);
            float dyv[32], l2 = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float d = 0.f;
                if (k < 13) {
                    const float e = __fsub_rn(y[k] + __ldg(a.bias + 512 + k), tgt[k]);
                    l2 += e * e;
                    d = sc * e;
                }
                dyv[k] = d;
                dyv[16 + k] = 0.f;
            }
#pragma unroll
            for (int k = 0; k < 16; k += 4)
                *reinterpret_cast<float4*>(a.dy + (size_t)b * 16 + k) = make_float4(dyv[k], dyv[k + 1], dyv[k + 2], dyv[k + 3]);
#pragma unroll
            for (int k = 0; k < 16; ++k) st_img(a.dz3T, 16, k, b, dyv[k]);
            const float col = warp_rs32(dyv);  // lane l: warp sum of dY column l
            if (lane < 16) a.db_part[((size_t)tile * 4 + q) * NBIAS + 512 + lane] = col;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
            if (lane == 0) red[q] = l2;
        }
        __syncthreads();
        if (tid == 0) a.loss_part[tile] = ((red[0] + red[1]) + red[2]) + red[3];
    }
    if (!ok && tid == 0) atomicOr(a.status, 2);
    tile_epilogue(tmem);
}

// ------------------------------------------------------------- backward (data)
__global__ void __launch_bounds__(256, 1) k_surr_bwd_train(const TrainArgs a) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    uint8_t* sm = smraw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* imgB = sm;                     // W3^T (cols 0..15) + dY tile (rows 0..127, cols 16..31)
    uint8_t* imgW2T = sm + IMG_A;
    uint8_t* imgG = sm + IMG_A + IMG_W2;    // dZ2 tile
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + SMEM_TR);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t q = warp & 3, half = warp >> 2, r = 32u * q + lane;
    uint32_t tmem;
    bool ok = tile_prologue(sm, SMEM_TR, a.imgB, IMG_A, a.imgW2T, IMG_W2, IMG_A, a.status, tmem);
    const uint32_t sB = smem_u32(imgB), sW2T = smem_u32(imgW2T), sG = smem_u32(imgG);
    const uint32_t tq = tmem + ((32u * q) << 16);
    const int tile = blockIdx.x;
    const uint32_t b = (uint32_t)tile * 128u + r;
    uint32_t ph = 0;
    if (tid < 128) {
        float d[16];
#pragma unroll
        for (int k = 0; k < 16; k += 4) {
            const float4 v4 = *reinterpret_cast<const float4*>(a.dy + (size_t)b * 16 + k);
            d[k] = v4.x; d[k + 1] = v4.y; d[k + 2] = v4.z; d[k + 3] = v4.w;
        }
        uint32_t p[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) p[i] = pack_bf16(d[2 * i], d[2 * i + 1]);
        st_chunk_t(imgB, r, 2, make_uint4(p[0], p[1], p[2], p[3]));
        st_chunk_t(imgB, r, 3, make_uint4(p[4], p[5], p[6], p[7]));
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (ok && tid == 0) {  // dH2 = dY (K = 16) * W3 -> columns [0, 256)
        tc_fence_after();
        mma_bf16(tmem, desc_sw128(sB + 32), desc_sw128(sB), idesc_bf16(128, 256), 0);
        mma_commit(&bars[1]);
    }
    for (int layer = 1; layer >= 0 && ok; --layer) {
        if (!(ok = sync_wait_t(&bars[1], ph))) break;
        tc_fence_after();
        const float* z = layer == 1 ? a.z2 : a.z1;
        uint8_t* dT = layer == 1 ? a.dz2T : a.dz1T;
        const uint32_t dcol = layer == 1 ? 0u : 256u;
        const uint32_t bslot = layer == 1 ? 256u : 0u;
#pragma unroll 1
        for (uint32_t c = 0; c < 4; ++c) {
            const uint32_t col0 = half * 128 + 32 * c;
            float v[32];
            tmem_ld32(tq + dcol + col0, v);
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
                const float4 z4 = *reinterpret_cast<const float4*>(z + (size_t)b * 256 + col0 + i);
                v[i] *= dsilu_t(z4.x);
                v[i + 1] *= dsilu_t(z4.y);
                v[i + 2] *= dsilu_t(z4.z);
                v[i + 3] *= dsilu_t(z4.w);
            }
            uint32_t p[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) p[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            if (layer == 1) {
                uint8_t* blk = imgG + (col0 >> 6) * 16384u;
                const uint32_t c0 = (col0 & 63u) >> 3;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    st_chunk_t(blk, r, c0 + j, make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]));
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&p[i]);
                *reinterpret_cast<__nv_bfloat16*>(dT + img_off(col0 + 2 * i, b, 256)) = h2.x;
                *reinterpret_cast<__nv_bfloat16*>(dT + img_off(col0 + 2 * i + 1, b, 256)) = h2.y;
            }
            const float cs = warp_rs32(v);  // lane l: column col0 + l summed over the warp's rows
            a.db_part[((size_t)tile * 4 + q) * NBIAS + bslot + col0 + lane] = cs;
        }
        if (layer == 1) {
            tc_fence_before();
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {  // dH1 = dZ2 * W2 -> columns [256, 512)
                tc_fence_after();
#pragma unroll
                for (uint32_t ks = 0; ks < 16; ++ks) {
                    const uint32_t kb = ks >> 2, off = (ks & 3) * 32;
                    mma_bf16(tmem + 256, desc_sw128(sG + kb * 16384 + off), desc_sw128(sW2T + kb * 32768 + off),
                             idesc_bf16(128, 256), ks);
                }
                mma_commit(&bars[1]);
            }
        }
    }
    if (!ok && tid == 0) atomicOr(a.status, 2);
    tile_epilogue(tmem);
}

// ------------------------------------------------------------- weight gradients
// CTA (g, m-tile, split): D[128 x N] = sum over its K-blocks (64 batch rows
// each) of A-tile * B^T; g = 0: dW1 (A dZ1^T, B X^T, N = 32), 1: dW2 (A dZ2^T,
// B H1^T, N = 256), 2: dW3^T (A H2^T, B dY^T, N = 16).
__global__ void __launch_bounds__(128, 1) k_surr_wgrad(const TrainArgs a) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    uint8_t* sm = smraw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + WG_STAGES * WG_STAGE);
    uint64_t* empty = full + WG_STAGES;
    uint64_t* done = empty + WG_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per_g = 2 * a.splits;
    const int g = blockIdx.x / per_g, rem = blockIdx.x - g * per_g, mt = rem / a.splits, sp = rem - mt * a.splits;
    const uint8_t* Aimg = g == 0 ? a.dz1T : (g == 1 ? a.dz2T : a.h2T);
    const uint8_t* Bimg = g == 0 ? a.xT : (g == 1 ? a.h1T : a.dz3T);
    const uint32_t N = g == 0 ? 32u : (g == 1 ? 256u : 16u);
    const int nkb = a.B / 64, kb0 = sp * nkb / a.splits, kb1 = (sp + 1) * nkb / a.splits;
    const uint32_t bbytes = N * 128u;
    if (tid == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t sbase = smem_u32(sm);
    bool ok = true;  // meaningful on thread 0, the producer and MMA issuer
    if (tid == 0) {
        const int n = kb1 - kb0;
        auto issue = [&](int i) {  // K-block kb0 + i into stage i % STAGES
            const int s = i % WG_STAGES, kb = kb0 + i;
            mbar_expect_tx(&full[s], 16384u + bbytes);
            bulk_g2s(sm + s * WG_STAGE, Aimg + (size_t)kb * 256 * 128 + (size_t)mt * 128 * 128, 16384u, &full[s]);
            bulk_g2s(sm + s * WG_STAGE + 16384, Bimg + (size_t)kb * bbytes, bbytes, &full[s]);
        };
        for (int i = 0; i < n && i < WG_STAGES; ++i) issue(i);
        for (int i = 0; i < n && ok; ++i) {
            const int s = i % WG_STAGES;
            const uint32_t par = (uint32_t)(i / WG_STAGES) & 1u;
            if (!(ok = mbar_wait(&full[s], par))) break;
            tc_fence_after();
            const uint32_t sa = sbase + s * WG_STAGE, sb = sa + 16384;
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), idesc_bf16(128, N), (i > 0 || kk > 0));
            mma_commit(&empty[s]);
            if (i + WG_STAGES < n) {
                if (!(ok = mbar_wait(&empty[s], par))) break;
                issue(i + WG_STAGES);
            }
        }
        if (n > 0) mma_commit(done);
        else mbar_expect_tx(done, 0);  // nothing to do: complete the phase
    }
    const bool all_ok = __syncthreads_and(mbar_wait(done, 0) && ok) != 0;
    tc_fence_after();
    if (all_ok) {
        const uint32_t tq = tmem + ((32u * (uint32_t)warp) << 16);
        const size_t row = (size_t)mt * 128 + 32 * warp + lane;
        size_t base;
        if (g == 0) base = 0;
        else if (g == 1) base = (size_t)a.splits * 256 * 32;
        else base = (size_t)a.splits * 256 * (32 + 256);
        float* out = a.wpart + base + ((size_t)sp * 256 + row) * N;
        for (uint32_t n0 = 0; n0 < N; n0 += 16) {
            float v[16];
            tmem_ld16(tq + n0, v);
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4*>(out + n0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    } else if (tid == 0) {
        atomicOr(a.status, 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// ------------------------------------------------------------- Adam
__global__ void k_surr_adam(const TrainArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ntiles = a.B / 128;
    if (i == 0 && a.loss) {
        float s = 0.f;
        for (int t = 0; t < ntiles; ++t) s += a.loss_part[t];
        *a.loss = s / (float)(a.B * NOUT);
    }
    if (i >= NPARAM) return;
    const int S = a.splits;
    const float* w1 = a.wpart;
    const float* w2 = w1 + (size_t)S * 256 * 32;
    const float* w3 = w2 + (size_t)S * 256 * 256;
    auto bias_sum = [&](int slot) {
        float s = 0.f;
        for (int t = 0; t < ntiles; ++t)
            for (int q = 0; q < 4; ++q) s += a.db_part[((size_t)t * 4 + q) * NBIAS + slot];
        return s;
    };
    float g = 0.f;
    if (i < OFF_B1) {
        const int o = i / NIN, k = i - o * NIN;
        for (int s = 0; s < S; ++s) g += w1[((size_t)s * 256 + o) * 32 + k];
    } else if (i < OFF_W2) {
        g = bias_sum(i - OFF_B1);
    } else if (i < OFF_B2) {
        const int j = i - OFF_W2, o = j >> 8, k = j & 255;
        for (int s = 0; s < S; ++s) g += w2[((size_t)s * 256 + o) * 256 + k];
    } else if (i < OFF_W3) {
        g = bias_sum(256 + i - OFF_B2);
    } else if (i < OFF_B3) {
        const int j = i - OFF_W3, o = j >> 8, k = j & 255;
        for (int s = 0; s < S; ++s) g += w3[((size_t)s * 256 + k) * 16 + o];
    } else {
        g = bias_sum(512 + i - OFF_B3);
    }
    if (a.grads) a.grads[i] = g;
    if (!a.apply) return;
    const float m = __fadd_rn(__fmul_rn(a.beta1, a.m[i]), __fmul_rn(1.f - a.beta1, g));
    const float v = __fadd_rn(__fmul_rn(a.beta2, a.v[i]), __fmul_rn(__fmul_rn(1.f - a.beta2, g), g));
    const float mh = __fmul_rn(m, a.c1), vh = __fmul_rn(v, a.c2);
    const float w = __fsub_rn(a.P[i], __fdiv_rn(__fmul_rn(a.lr, mh), __fadd_rn(sqrtf(vh), a.eps)));
    a.m[i] = m;
    a.v[i] = v;
    a.P[i] = w;
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    if (i < OFF_B1) {
        const int o = i / NIN, k = i - o * NIN;
        *reinterpret_cast<__nv_bfloat16*>(a.imgA + img_off(o, k, 256)) = b;
    } else if (i < OFF_W2) {
        a.bias[i - OFF_B1] = w;
    } else if (i < OFF_B2) {
        const int j = i - OFF_W2, o = j >> 8, k = j & 255;
        *reinterpret_cast<__nv_bfloat16*>(a.imgW2 + img_off(o, k, 256)) = b;
        *reinterpret_cast<__nv_bfloat16*>(a.imgW2T + img_off(k, o, 256)) = b;
    } else if (i < OFF_W3) {
        a.bias[256 + i - OFF_B2] = w;
    } else if (i < OFF_B3) {
        const int j = i - OFF_W3, o = j >> 8, k = j & 255, piece = k >> 5;
        *reinterpret_cast<__nv_bfloat16*>(a.imgA + img_off(128 + 16 * piece + o, 32 + (k & 31), 256)) = b;
        *reinterpret_cast<__nv_bfloat16*>(a.imgB + img_off(k, o, 256)) = b;
    } else {
        a.bias[512 + i - OFF_B3] = w;
    }
}

// ------------------------------------------------------------- launcher
// One optimisation step (apply = 0: gradients only).  B a multiple of 128.
cudaError_t launch_surr_train(const TrainArgs& a, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_surr_fwd_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TR_LAUNCH)) ||
        (e = cudaFuncSetAttribute(k_surr_bwd_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TR_LAUNCH)) ||
        (e = cudaFuncSetAttribute(k_surr_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_WG_LAUNCH)))
        return e;
    const int tiles = a.B / 128;
    k_surr_fwd_train<<<tiles, 256, SMEM_TR_LAUNCH, st>>>(a);
    if ((e = cudaGetLastError())) return e;
    k_surr_bwd_train<<<tiles, 256, SMEM_TR_LAUNCH, st>>>(a);
    if ((e = cudaGetLastError())) return e;
    k_surr_wgrad<<<3 * 2 * a.splits, 128, SMEM_WG_LAUNCH, st>>>(a);
    if ((e = cudaGetLastError())) return e;
    k_surr_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sg
