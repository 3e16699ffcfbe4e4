// gemm.cuh -- a streamed-K bf16 GEMM on the tensor cores (tcgen05, fp32
// accumulators in tensor memory), operands in the 128-byte swizzled image
// layout of umma.cuh, with the epilogues of the closed-loop policy.
//
//   D[M x N] = A[M x K] * B[N x K]^T
//
// A is an image of RA rows (RA a multiple of 128, rows beyond M zero), B an
// image of RB rows (RB >= N), both with K padded to whole 64-column blocks.
// CTA (m-tile of 128 rows, n-tile of up to 256 columns, K split) streams its
// K-blocks through a 4-stage ring of shared-memory stages filled by 1D bulk
// copies (one per operand tile: a K-block's rows are contiguous in an
// image), one thread issues the MMAs, four warps read the accumulator.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace gm {

enum Epilogue {
    EPI_STORE = 0,    // fp32 C[split][M][ldc] (split-K partials when splits > 1)
    EPI_POLICY = 1,   // policy layer 1: z = D + bias -> z_out [M][256] fp32, bf16(silu(z)) -> h_out [M][256]
    EPI_OBS_GRAD = 2  // observation cotangent: column n to g_f [M][16] (n < 16), g_cam [M][Rc] * cam_scale,
                      // g_lid [M][Rl] * lid_scale (the rest)
};

struct GemmArgs {
    const uint8_t* A;
    const uint8_t* B;
    int RA, RB;       // image rows
    int M, N, nkb;    // problem rows, columns, K-blocks of 64
    int splits;       // K splits (grid z)
    int epi;
    float* C;         // EPI_STORE
    int ldc;
    const float* bias;       // EPI_POLICY
    float* z_out;
    uint16_t* h_out;         // bf16 bits
    float *g_f, *g_cam, *g_lid;  // EPI_OBS_GRAD
    int Rc, Rl;
    float cam_scale, lid_scale;
    int* status;
};

// Grid: (ceil(M / 128), ceil(N / 256), splits); N a multiple of 16.
cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t st);

}  // namespace gm
