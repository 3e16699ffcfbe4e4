// peak.cu -- measured FP32-pipe issue rate of this GPU: the denominator of
// the ray cast's roofline, taken at the clock the GPU runs at.
//
// Every thread runs kChains independent multiply-add chains (enough
// independent work to hide the FMA latency) for `iters` rounds; the grid
// fills every SM several times over.  Two variants: scalar FMA (one
// instruction per lane and FMA) and packed pairs (one instruction per lane
// and two FMAs).  The chains stay bounded (x -> 0.75 x + 0.25 converges to
// 1), and their sum is written out so that no FMA can be dropped.
#include <cuda_runtime.h>

#include "diffsim.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.001f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ffma2(float* out, int iters, float a, float b) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(0.001f * (threadIdx.x + c), 0.002f * c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int sim_fp32_issue_rate(float* scratch, int64_t scratch_floats, double* fma_per_s, double* ffma2_per_s,
                                   sim_stream_t stream) {
    if (!scratch || !fma_per_s) return SIM_ERR_NULL_PTR;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SIM_ERR_CUDA;
    const int block = 256, grid = nsm * 8;
    if (scratch_floats < (int64_t)grid * block) return SIM_ERR_SIZE;
    const int iters = 4096;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SIM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SIM_ERR_CUDA;
    }
    int rc = SIM_OK;
    for (int variant = 0; variant < 2 && rc == SIM_OK; ++variant) {
        double* dst = variant == 0 ? fma_per_s : ffma2_per_s;
        if (!dst) continue;
        float best = 0.f;
        for (int rep = 0; rep < 4 && rc == SIM_OK; ++rep) {  // first pass warms up; keep the fastest
            cudaEventRecord(e0, st);
            if (variant == 0) k_ffma<<<grid, block, 0, st>>>(scratch, iters, 0.75f, 0.25f);
            else k_ffma2<<<grid, block, 0, st>>>(scratch, iters, 0.75f, 0.25f);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = SIM_ERR_CUDA;
                break;
            }
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        if (rc == SIM_OK) {
            const double fmas = (double)grid * block * iters * 8.0 * kChains * (variant == 0 ? 1.0 : 2.0);
            *dst = fmas / (best * 1e-3);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
