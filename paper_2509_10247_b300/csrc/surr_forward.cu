// surr_forward.cu -- surrogate MLP forward pass and rollout on the tensor
// cores (tcgen05, accumulators in tensor memory), weight packing, and the
// normalisation statistics of a transition set.
//
// Rollout: a persistent CTA per SM takes tiles of 128 environments; the
// weights stay in shared memory for the CTA's lifetime (one bulk copy), the
// tile's states stay in registers for all T steps.  Per step: the input tile
// X (bf16) is formed in shared memory, then three chained MMAs (M = 128, N =
// 256 / 256 / 16) with epilogues between them (bias, SiLU, bf16, back into
// shared memory as the next A operand); the last epilogue applies the
// residual, renormalises the quaternion, or takes the plain rigid-body step
// where the inputs left the trained range.
#include "surr_kernels.cuh"
#include "umma.cuh"

namespace sg {
using namespace um;

constexpr uint32_t SMEM_FWD = IMG_A + IMG_W2 + IMG_H;  // 224 KiB of images
constexpr uint32_t SMEM_FWD_LAUNCH = SMEM_FWD + 1024 + 64;  // + alignment slack + barriers

// SiLU with the fast exponential and division (a few ulp of fp32; the result
// is rounded to bf16, 2^-8 relative, right after).
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// One 16-byte chunk (8 bf16, columns 8c .. 8c+7 of a K-block) of row r.
__device__ __forceinline__ void st_chunk(uint8_t* blk, uint32_t r, uint32_t c, uint4 v) {
    *reinterpret_cast<uint4*>(blk + r * 128u + (((c ^ r) & 7u) << 4)) = v;
}

// Hidden-layer epilogue of 32 accumulator columns [col0, col0 + 32) of the
// thread's row r: bias, SiLU, bf16, into the activation image (256 columns).
__device__ __forceinline__ void epi_hidden(uint32_t taddr, const float* bias, uint32_t col0, uint8_t* img,
                                           uint32_t r) {
    float v[32];
    tmem_ld32(taddr, v);
    uint32_t p[16];
    const float4* b4 = reinterpret_cast<const float4*>(bias + col0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 b = __ldg(b4 + i);
        p[2 * i] = pack_bf16(silu_f(v[4 * i] + b.x), silu_f(v[4 * i + 1] + b.y));
        p[2 * i + 1] = pack_bf16(silu_f(v[4 * i + 2] + b.z), silu_f(v[4 * i + 3] + b.w));
    }
    uint8_t* blk = img + (col0 >> 6) * 16384u;
    const uint32_t c0 = (col0 & 63u) >> 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) st_chunk(blk, r, c0 + j, make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]));
}

__device__ __forceinline__ bool sync_wait(uint64_t* bar, uint32_t& ph) {
    const bool ok = __syncthreads_and(mbar_wait(bar, ph)) != 0;
    ph ^= 1u;
    return ok;
}

__global__ void __launch_bounds__(256, 1) k_surr_fwd(const SurrArgs a) {
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    uint8_t* sm = smraw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* imgA = sm;
    uint8_t* imgW2 = sm + IMG_A;
    uint8_t* imgH = sm + IMG_A + IMG_W2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + SMEM_FWD);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SMEM_FWD + 16);
    int* sflag = reinterpret_cast<int*>(sm + SMEM_FWD + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t q = warp & 3, half = warp >> 2;
    const uint32_t r = 32u * q + lane;  // tile row of this thread (== tid on warps 0..3)

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_barrier_init();
        *sflag = 1;
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(tslot, 512);
    if (tid == 0) {
        mbar_expect_tx(&bars[0], IMG_A + IMG_W2);
        bulk_g2s(imgA, a.imgA, IMG_A, &bars[0]);
        bulk_g2s(imgW2, a.imgW2, IMG_W2, &bars[0]);
        if (!mbar_wait(&bars[0], 0)) {
            atomicOr(a.status, 2);
            *sflag = 0;
            mbar_wait(&bars[0], 0);  // a second bounded chance for the copies in flight
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = *sflag != 0;

    const uint32_t sA = smem_u32(imgA), sW2 = smem_u32(imgW2), sH = smem_u32(imgH);
    const uint32_t id256 = idesc_bf16(128, 256), id16 = idesc_bf16(128, 16);
    const uint32_t tq = tmem + ((32u * q) << 16);  // this warp's lane quarter
    const float* st = a.stats;
    const bool own = tid < 128;
    const int T = a.mode == 0 ? a.T : 1;
    const int ntiles = (a.N + 127) / 128;
    uint32_t ph = 0;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int row = tile * 128 + (int)r;
        const bool valid = own && row < a.N;
        float s[13];
#pragma unroll
        for (int k = 0; k < 13; ++k) s[k] = (valid && a.mode == 0) ? a.s0[(size_t)row * 13 + k] : 0.f;
        if (valid && a.mode == 0 && a.states)
#pragma unroll
            for (int k = 0; k < 13; ++k) a.states[(size_t)row * 13 + k] = s[k];
        for (int t = 0; t < T; ++t) {
            float act[4] = {0.f, 0.f, 0.f, 0.f};
            bool inr = true;
            if (own) {
                float x[17];
                if (a.mode == 0) {
#pragma unroll
                    for (int k = 0; k < 13; ++k) x[k] = s[k];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        act[k] = valid ? a.actions[((size_t)t * a.N + row) * 4 + k] : 0.f;
                        x[13 + k] = ds::clip1(act[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 17; ++k) x[k] = valid ? a.X[(size_t)row * 17 + k] : 0.f;
#pragma unroll
                    for (int k = 13; k < 17; ++k) x[k] = ds::clip1(x[k]);
                }
                float xh[32];
#pragma unroll
                for (int k = 0; k < 17; ++k) {
                    const float lo = st[ST_LOX + k], hi = st[ST_HIX + k], m = a.margin > 0.f ? a.margin * (hi - lo) : 0.f;
                    inr = inr && x[k] >= lo - m && x[k] <= hi + m;
                    xh[k] = __fmul_rn(__fsub_rn(x[k], st[ST_MUX + k]), st[ST_RSX + k]);
                }
#pragma unroll
                for (int k = 17; k < 32; ++k) xh[k] = 0.f;
                uint32_t p[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) p[i] = pack_bf16(xh[2 * i], xh[2 * i + 1]);
                // input tile: columns 32..63 (chunks 4..7) of image A's rows 0..127
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    st_chunk(imgA, r, 4 + j, make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]));
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            // layer 1: D[0, 256) = X (K = 32) * W1^T
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (uint32_t ks = 0; ks < 2; ++ks)
                    mma_bf16(tmem, desc_sw128(sA + 64 + 32 * ks), desc_sw128(sA + 32 * ks), id256, ks);
                mma_commit(&bars[1]);
            }
            if (!(ok = sync_wait(&bars[1], ph))) break;
            tc_fence_after();
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c) {
                const uint32_t col0 = half * 128 + 32 * c;
                epi_hidden(tq + col0, a.bias, col0, imgH, r);
            }
            tc_fence_before();
            fence_async_smem();
            __syncthreads();
            // layer 2: D[256, 512) = H1 * W2^T (K = 256)
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (uint32_t ks = 0; ks < 16; ++ks) {
                    const uint32_t kb = ks >> 2, off = (ks & 3) * 32;
                    mma_bf16(tmem + 256, desc_sw128(sH + kb * 16384 + off), desc_sw128(sW2 + kb * 32768 + off), id256,
                             ks);
                }
                mma_commit(&bars[1]);
            }
            if (!(ok = sync_wait(&bars[1], ph))) break;
            tc_fence_after();
#pragma unroll
            for (uint32_t c = 0; c < 4; ++c) {
                const uint32_t col0 = half * 128 + 32 * c;
                epi_hidden(tq + 256 + col0, a.bias + 256, col0, imgH, r);
            }
            tc_fence_before();
            fence_async_smem();
            __syncthreads();
            // layer 3: D[0, 16) = H2 * W3^T (K = 256; W3 pieces in image A)
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (uint32_t ks = 0; ks < 16; ++ks) {
                    const uint32_t adr = sH + (ks >> 2) * 16384 + (ks & 3) * 32;
                    const uint32_t bdr = sA + (128 + 16 * (ks >> 1)) * 128 + 64 + (ks & 1) * 32;
                    mma_bf16(tmem, desc_sw128(adr), desc_sw128(bdr), id16, ks);
                }
                mma_commit(&bars[1]);
            }
            if (!(ok = sync_wait(&bars[1], ph))) break;
            tc_fence_after();
            if (own) {
                float y[16];
                tmem_ld16(tq, y);
#pragma unroll
                for (int k = 0; k < 13; ++k) y[k] += __ldg(a.bias + 512 + k);
                if (valid && a.mode == 1) {
#pragma unroll
                    for (int k = 0; k < 13; ++k) a.Y[(size_t)row * 13 + k] = y[k];
                } else if (valid) {
                    float sp[16];
                    if (inr) {
#pragma unroll
                        for (int k = 0; k < 13; ++k)
                            sp[k] = __fadd_rn(s[k], __fadd_rn(__fmul_rn(st[ST_SDD + k], y[k]), st[ST_MUD + k]));
                        const float nq = sqrtf(sp[3] * sp[3] + sp[4] * sp[4] + sp[5] * sp[5] + sp[6] * sp[6]);
#pragma unroll
                        for (int k = 3; k < 7; ++k) sp[k] = sp[k] / nq;
                    } else {
                        ds::rb_step(a.c, s, act, sp);
                    }
#pragma unroll
                    for (int k = 0; k < 13; ++k) s[k] = sp[k];
                    if (a.states)
#pragma unroll
                        for (int k = 0; k < 13; ++k) a.states[((size_t)(t + 1) * a.N + row) * 13 + k] = s[k];
                    if (a.fallback) a.fallback[(size_t)t * a.N + row] = inr ? 0 : 1;
                    bool fin = true;
#pragma unroll
                    for (int k = 0; k < 13; ++k) fin = fin && isfinite(s[k]);
                    if (!fin) atomicOr(a.status, 1);
                }
            }
            tc_fence_before();
            __syncthreads();
        }
        if (ok && valid && a.mode == 0 && a.sT)
#pragma unroll
            for (int k = 0; k < 13; ++k) a.sT[(size_t)row * 13 + k] = s[k];
    }
    if (!ok && tid == 0) atomicOr(a.status, 2);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Master parameters (fp32) -> bf16 images and the fp32 bias block.  The
// images and the bias block are zeroed before (padding stays zero).
__global__ void k_surr_pack(const float* P, uint8_t* imgA, uint8_t* imgW2, uint8_t* imgB, uint8_t* imgW2T,
                            float* bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float w = P[i];
    const __nv_bfloat16 b = __float2bfloat16_rn(w);
    if (i < OFF_B1) {
        const int o = i / NIN, k = i - o * NIN;
        *reinterpret_cast<__nv_bfloat16*>(imgA + img_off(o, k, 256)) = b;
    } else if (i < OFF_W2) {
        bias[i - OFF_B1] = w;
    } else if (i < OFF_B2) {
        const int j = i - OFF_W2, o = j >> 8, k = j & 255;
        *reinterpret_cast<__nv_bfloat16*>(imgW2 + img_off(o, k, 256)) = b;
        *reinterpret_cast<__nv_bfloat16*>(imgW2T + img_off(k, o, 256)) = b;
    } else if (i < OFF_W3) {
        bias[256 + i - OFF_B2] = w;
    } else if (i < OFF_B3) {
        const int j = i - OFF_W3, o = j >> 8, k = j & 255, piece = k >> 5;
        *reinterpret_cast<__nv_bfloat16*>(imgA + img_off(128 + 16 * piece + o, 32 + (k & 31), 256)) = b;
        *reinterpret_cast<__nv_bfloat16*>(imgB + img_off(k, o, 256)) = b;
    } else {
        bias[512 + i - OFF_B3] = w;
    }
}

// Statistics of a transition set, pass 1: block b reduces rows [b * chunk,
// (b + 1) * chunk) into part[b][30][4] = (sum, sum of squares, min, max) of
// the 17 inputs (actions clipped) and the 13 residuals s1 - s.  Thread
// (feature f = tid & 31, row group g = tid >> 5) strides rows by 8; the 8
// groups combine in a fixed order.
__global__ void __launch_bounds__(256) k_surr_stats_part(const float* X, const float* S1, long long n,
                                                         long long chunk, double* part) {
    __shared__ double sh[8][30][4];
    const int f = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long r0 = (long long)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    double s1 = 0.0, s2 = 0.0, mn = CUDART_INF, mx = -CUDART_INF;
    if (f < 30)
        for (long long r = r0 + g; r < r1; r += 8) {
            float v;
            if (f < NIN) {
                v = X[r * NIN + f];
                if (f >= 13) v = ds::clip1(v);
            } else {
                v = __fsub_rn(S1[r * NOUT + (f - NIN)], X[r * NIN + (f - NIN)]);
            }
            const double d = v;
            s1 += d;
            s2 += d * d;
            mn = fmin(mn, d);
            mx = fmax(mx, d);
        }
    if (f < 30) {
        sh[g][f][0] = s1; sh[g][f][1] = s2; sh[g][f][2] = mn; sh[g][f][3] = mx;
    }
    __syncthreads();
    if (threadIdx.x < 30) {
        double a1 = 0.0, a2 = 0.0, a3 = CUDART_INF, a4 = -CUDART_INF;
        for (int k = 0; k < 8; ++k) {
            a1 += sh[k][threadIdx.x][0];
            a2 += sh[k][threadIdx.x][1];
            a3 = fmin(a3, sh[k][threadIdx.x][2]);
            a4 = fmax(a4, sh[k][threadIdx.x][3]);
        }
        double* o = part + ((size_t)blockIdx.x * 30 + threadIdx.x) * 4;
        o[0] = a1; o[1] = a2; o[2] = a3; o[3] = a4;
    }
}

// Pass 2 (one block): combine the partials in block order into the
// statistics vector (mu_x, rs_x, lo_x, hi_x, mu_d, sd_d, rs_d).
__global__ void k_surr_stats_final(const double* part, int nblk, long long n, float* stats) {
    const int f = threadIdx.x;
    if (f >= 30) return;
    double a1 = 0.0, a2 = 0.0, mn = CUDART_INF, mx = -CUDART_INF;
    for (int b = 0; b < nblk; ++b) {
        const double* p = part + ((size_t)b * 30 + f) * 4;
        a1 += p[0]; a2 += p[1]; mn = fmin(mn, p[2]); mx = fmax(mx, p[3]);
    }
    const double mu = a1 / (double)n;
    const double sd = sqrt(fmax(a2 / (double)n - mu * mu, 0.0));
    const double rs = sd < 1e-6 ? 1.0 : 1.0 / sd;
    if (f < NIN) {
        stats[ST_MUX + f] = (float)mu;
        stats[ST_RSX + f] = (float)rs;
        stats[ST_LOX + f] = (float)mn;
        stats[ST_HIX + f] = (float)mx;
    } else {
        const int k = f - NIN;
        stats[ST_MUD + k] = (float)mu;
        stats[ST_SDD + k] = (float)sd;
        stats[ST_RSD + k] = (float)rs;
    }
}

// ------------------------------------------------------------- launchers
cudaError_t launch_surr_fwd(const SurrArgs& a, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_surr_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_FWD_LAUNCH);
    if (e != cudaSuccess) return e;
    const int ntiles = (a.N + 127) / 128;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    if (grid < 1) return cudaSuccess;
    k_surr_fwd<<<grid, 256, SMEM_FWD_LAUNCH, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_surr_pack(const float* P, uint8_t* imgA, uint8_t* imgW2, uint8_t* imgB, uint8_t* imgW2T,
                             float* bias, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(imgA, 0, IMG_A, st)) || (e = cudaMemsetAsync(imgW2, 0, IMG_W2, st)) ||
        (e = cudaMemsetAsync(imgB, 0, IMG_A, st)) || (e = cudaMemsetAsync(imgW2T, 0, IMG_W2, st)) ||
        (e = cudaMemsetAsync(bias, 0, NBIAS * sizeof(float), st)))
        return e;
    k_surr_pack<<<(NPARAM + 255) / 256, 256, 0, st>>>(P, imgA, imgW2, imgB, imgW2T, bias);
    return cudaGetLastError();
}

cudaError_t launch_surr_stats(const float* X, const float* S1, long long n, double* part, int nblk, float* stats,
                              cudaStream_t st) {
    const long long chunk = (n + nblk - 1) / nblk;
    k_surr_stats_part<<<nblk, 256, 0, st>>>(X, S1, n, chunk, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_surr_stats_final<<<1, 32, 0, st>>>(part, nblk, n, stats);
    return cudaGetLastError();
}

}  // namespace sg
