// gemm.cu -- streamed-K tcgen05 GEMM with the closed-loop policy's epilogues
// (see gemm.cuh).
#include <cuda_bf16.h>

#include "gemm.cuh"
#include "umma.cuh"

namespace gm {
using namespace um;

constexpr uint32_t A_TILE = 16384;
__host__ __device__ constexpr uint32_t stage_bytes(int bn) { return A_TILE + (uint32_t)bn * 128u; }
__host__ __device__ constexpr uint32_t smem_launch(int stages, int bn) {
    return stages * stage_bytes(bn) + 1024 + 128;
}

// STAGES: depth of the K ring; BN: columns of the n-tile (and of the tensor
// memory the CTA holds).  A long K (the policy's layer 1, the weight
// gradient) keeps four stages of 256-column tiles in flight; a short K (the
// observation cotangent, K = 256) takes two stages of 128 columns, so three
// CTAs share an SM (3 x 128 tensor-memory columns) and their epilogues
// overlap one another's loads and MMAs.
template <int STAGES, int BN>
__global__ void __launch_bounds__(128, 1) k_gemm(const GemmArgs a) {
    constexpr uint32_t STAGE = stage_bytes(BN);
    extern __shared__ __align__(1024) uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    uint8_t* sm = smraw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, nt = blockIdx.y, sp = blockIdx.z;
    const int n0 = nt * BN;
    const uint32_t Nt = (uint32_t)min(BN, a.N - n0);
    const int kb0 = (int)((long long)sp * a.nkb / a.splits), kb1 = (int)((long long)(sp + 1) * a.nkb / a.splits);
    const uint32_t bbytes = Nt * 128u;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(tslot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t sbase = smem_u32(sm);
    bool ok = true;  // producer / MMA issuer (thread 0)
    if (tid == 0) {
        const int n = kb1 - kb0;
        auto issue = [&](int i) {
            const int s = i % STAGES;
            const size_t kb = (size_t)(kb0 + i);
            mbar_expect_tx(&full[s], A_TILE + bbytes);
            bulk_g2s(sm + s * STAGE, a.A + kb * (size_t)a.RA * 128 + (size_t)mt * 128 * 128, A_TILE, &full[s]);
            bulk_g2s(sm + s * STAGE + A_TILE, a.B + kb * (size_t)a.RB * 128 + (size_t)n0 * 128, bbytes, &full[s]);
        };
        for (int i = 0; i < n && i < STAGES; ++i) issue(i);
        const uint32_t idesc = idesc_bf16(128, Nt);
        for (int i = 0; i < n && ok; ++i) {
            const int s = i % STAGES;
            const uint32_t par = (uint32_t)(i / STAGES) & 1u;
            if (!(ok = mbar_wait(&full[s], par))) break;
            tc_fence_after();
            const uint32_t sa = sbase + s * STAGE, sb = sa + A_TILE;
#pragma unroll
            for (uint32_t kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, desc_sw128(sa + 32 * kk), desc_sw128(sb + 32 * kk), idesc, (i > 0 || kk > 0));
            mma_commit(&empty[s]);
            if (i + STAGES < n) {
                if (!(ok = mbar_wait(&empty[s], par))) break;
                issue(i + STAGES);
            }
        }
        if (n > 0) mma_commit(done);
        else mbar_expect_tx(done, 0);
    }
    const bool all_ok = __syncthreads_and(mbar_wait(done, 0) && ok) != 0;
    tc_fence_after();
    const bool empty_k = kb1 <= kb0;  // no K-block: the accumulator holds nothing
    if (all_ok && a.epi == EPI_OBS_GRAD) {
        // Observation cotangent: 64 accumulator columns at a time go through
        // shared memory (the drained stage ring) so that the warp stores whole
        // row segments (32 lanes on consecutive columns of one row) instead of
        // one column per row.  Each warp stages and stores its own 32 rows.
        fence_async_smem();
        float* stg = reinterpret_cast<float*>(sm) + warp * 32 * 65;
        const uint32_t tq = tmem + ((32u * (uint32_t)warp) << 16);
        const int Rc = a.Rc, Rl = a.Rl;
        const bool vec4 = (Rc & 3) == 0 && (Rl & 3) == 0 && ((uintptr_t)a.g_f & 15) == 0 &&
                          ((uintptr_t)a.g_cam & 15) == 0 && ((uintptr_t)a.g_lid & 15) == 0;
        for (uint32_t c0 = 0; c0 < Nt; c0 += 64) {
            const uint32_t nc = min(64u, Nt - c0);
            for (uint32_t cc = 0; cc < nc; cc += 16) {
                float v[16];
                tmem_ld16(tq + c0 + cc, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) stg[lane * 65 + cc + i] = empty_k ? 0.f : v[i];
            }
            __syncwarp();
            if (vec4) {
                // two rows per pass, 16 lanes x 4 consecutive columns each:
                // 16-byte stores (every region starts at a multiple of 4)
                for (int it = 0; it < 16; ++it) {
                    const int rr = 2 * it + (lane >> 4), cp = (lane & 15) * 4;
                    const int row = mt * 128 + 32 * warp + rr;
                    if (row >= a.M || cp >= (int)nc) continue;
                    const int n = n0 + (int)c0 + cp;
                    float4 x = make_float4(stg[rr * 65 + cp], stg[rr * 65 + cp + 1], stg[rr * 65 + cp + 2],
                                           stg[rr * 65 + cp + 3]);
                    float* dst;
                    if (n < 16) dst = a.g_f + (size_t)row * 16 + n;
                    else if (n < 16 + Rc) {
                        dst = a.g_cam + (size_t)row * Rc + (n - 16);
                        x = make_float4(x.x * a.cam_scale, x.y * a.cam_scale, x.z * a.cam_scale, x.w * a.cam_scale);
                    } else if (n < 16 + Rc + Rl) {
                        dst = a.g_lid + (size_t)row * Rl + (n - 16 - Rc);
                        x = make_float4(x.x * a.lid_scale, x.y * a.lid_scale, x.z * a.lid_scale, x.w * a.lid_scale);
                    } else {
                        continue;
                    }
                    *reinterpret_cast<float4*>(dst) = x;
                }
            } else {
                for (int rr = 0; rr < 32; ++rr) {
                    const int row = mt * 128 + 32 * warp + rr;
                    if (row >= a.M) break;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int cp = lane + 32 * h;
                        if (cp >= (int)nc) continue;
                        const int n = n0 + (int)c0 + cp;
                        const float x = stg[rr * 65 + cp];
                        if (n < 16) a.g_f[(size_t)row * 16 + n] = x;
                        else if (n < 16 + Rc) a.g_cam[(size_t)row * Rc + (n - 16)] = x * a.cam_scale;
                        else if (n < 16 + Rc + Rl) a.g_lid[(size_t)row * Rl + (n - 16 - Rc)] = x * a.lid_scale;
                    }
                }
            }
            __syncwarp();
        }
    } else if (all_ok) {
        const uint32_t tq = tmem + ((32u * (uint32_t)warp) << 16);
        const int row = mt * 128 + 32 * warp + lane;
        const bool valid = row < a.M;
        for (uint32_t c0 = 0; c0 < Nt; c0 += 16) {
            float v[16];
            tmem_ld16(tq + c0, v);
            if (empty_k)
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            if (!valid) continue;
            const int col = n0 + (int)c0;
            if (a.epi == EPI_STORE) {
                float* out = a.C + ((size_t)sp * a.M + row) * a.ldc + col;
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(out + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            } else if (a.epi == EPI_POLICY) {
                float* zo = a.z_out + (size_t)row * 256 + col;
                uint32_t hp[8];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += __ldg(a.bias + col + i);
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(zo + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float s0 = __fdividef(v[2 * i], 1.f + __expf(-v[2 * i]));
                    const float s1 = __fdividef(v[2 * i + 1], 1.f + __expf(-v[2 * i + 1]));
                    hp[i] = pack_bf16(s0, s1);
                }
                uint4* ho = reinterpret_cast<uint4*>(a.h_out + (size_t)row * 256 + col);
                ho[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                ho[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = col + i;
                    if (n < 16) a.g_f[(size_t)row * 16 + n] = v[i];
                    else if (n < 16 + a.Rc) a.g_cam[(size_t)row * a.Rc + (n - 16)] = v[i] * a.cam_scale;
                    else if (n < 16 + a.Rc + a.Rl) a.g_lid[(size_t)row * a.Rl + (n - 16 - a.Rc)] = v[i] * a.lid_scale;
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(a.status, 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

template <int STAGES, int BN>
static cudaError_t launch_shape(const GemmArgs& a, cudaStream_t st) {
    const uint32_t smem = smem_launch(STAGES, BN);
    cudaError_t e = cudaFuncSetAttribute(k_gemm<STAGES, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.M + 127) / 128, (a.N + BN - 1) / BN, a.splits);
    k_gemm<STAGES, BN><<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t st) {
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    if (a.N % 16 || a.RA % 128 || a.RB < a.N || a.splits < 1) return cudaErrorInvalidValue;
    const int per_split = (a.nkb + a.splits - 1) / a.splits;
    if (per_split <= 8) return launch_shape<2, 128>(a, st);
    return launch_shape<4, 256>(a, st);
}

}  // namespace gm
