// surr_kernels.cuh -- shared declarations of the surrogate-MLP kernels.
//
// The surrogate of the rigid-body step (Eq. 1): inputs x = (s [13],
// clip(a) [4]), normalised xh = (x - mu_x) * rs_x, MLP 17 -> 256 -> 256 -> 13
// with SiLU, bf16 weights and activations, fp32 accumulation on the tensor
// cores (tcgen05, accumulators in tensor memory), output the normalised
// residual y; s' = s + (sd_d * y + mu_d), quaternion renormalised.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "sim_device.cuh"

namespace sg {

constexpr int NIN = 17, NHID = 256, NOUT = 13;
// parameter vector: W1 [256][17], b1 [256], W2 [256][256], b2 [256], W3 [13][256], b3 [13]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NHID * NIN, OFF_W2 = OFF_B1 + NHID, OFF_B2 = OFF_W2 + NHID * NHID,
              OFF_W3 = OFF_B2 + NHID, OFF_B3 = OFF_W3 + NOUT * NHID, NPARAM = OFF_B3 + NOUT;
// statistics: mu_x, rs_x, lo_x, hi_x [17], mu_d, sd_d, rs_d [13]
constexpr int ST_MUX = 0, ST_RSX = 17, ST_LOX = 34, ST_HIX = 51, ST_MUD = 68, ST_SDD = 81, ST_RSD = 94, NSTATS = 107;

// Weight images (bf16, 128-byte swizzled K-major, see umma.cuh):
//  A (32 KB, 256 rows x 64 columns): W1 in columns 0..31 of every row (17
//    real), the input tile X of the forward kernels in columns 32..63 of rows
//    0..127, and W3 in columns 32..63 of rows 128..255: piece j (j = 0..7)
//    holds W3[:, 32j .. 32j + 31] in rows 128 + 16j .. + 15 (13 real).
//  W2 (128 KB): W2 [256 out][256 in].
//  B (32 KB): W3^T [256 in] x columns 0..15 (13 real), the output-cotangent
//    tile dY of the backward kernel in columns 16..31 of rows 0..127.
//  W2T (128 KB): W2^T [256 in][256 out].
constexpr uint32_t IMG_A = 32768, IMG_W2 = 131072, IMG_H = 65536;
// bias block: b1 [256], b2 [256], b3 [16] (13 real)
constexpr int NBIAS = 528;

struct SurrArgs {
    const uint8_t* imgA;
    const uint8_t* imgW2;
    const float* bias;
    const float* stats;
    ds::Phys c;     // rigid-body parameters of the plain step taken outside the trained range
    float margin;   // trained-range margin, fraction of (hi - lo)
    int mode;       // 0 rollout, 1 forward of raw inputs X
    int N, T;
    const float* s0;       // [N][13] (rollout)
    const float* actions;  // [T][N][4] (rollout)
    const float* X;        // [N][17] (forward)
    float* Y;              // [N][13] normalised outputs (forward)
    float* states;         // [T+1][N][13] or null
    float* sT;             // [N][13] or null
    uint8_t* fallback;     // [T][N] or null
    int* status;
};

// Argument block of one training step (see surr_train.cu).
struct TrainArgs {
    uint8_t *imgA, *imgW2, *imgB, *imgW2T;
    float* bias;
    const float* stats;
    const float* X;   // [n][17] inputs (state, action)
    const float* S1;  // [n][13] next states
    const int* idx;   // [B] minibatch rows
    int B;
    float *z1, *z2;   // [B][256] pre-activations
    float* dy;        // [B][16] output cotangent
    uint8_t *xT, *h1T, *h2T, *dz3T, *dz2T, *dz1T;  // images [R][B]: R = 32, 256, 256, 16, 256, 256
    float* db_part;   // [B/128][4][NBIAS] column sums per tile and warp quarter
    float* loss_part; // [B/128]
    float* wpart;     // split partials: dW1 [S][256][32], dW2 [S][256][256], dW3^T [S][256][16]
    int splits;
    float *P, *m, *v, *grads, *loss;
    float lr, beta1, beta2, eps, c1, c2;
    int apply;
    int* status;
};

cudaError_t launch_surr_fwd(const SurrArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_surr_pack(const float* P, uint8_t* imgA, uint8_t* imgW2, uint8_t* imgB, uint8_t* imgW2T,
                             float* bias, cudaStream_t st);
cudaError_t launch_surr_stats(const float* X, const float* S1, long long n, double* part, int nblk, float* stats,
                              cudaStream_t st);
cudaError_t launch_surr_train(const TrainArgs& a, cudaStream_t st);

}  // namespace sg
