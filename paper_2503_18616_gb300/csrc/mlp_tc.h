// Warm-start network on tensor cores (internal to the library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ffsrl {

// BF16 weight tiles: W1 (64 x 16), W2 (64 x 64), W3 (16 x 64), K-major core-matrix layout.
constexpr int kMlpWeightBytes = (64 * 16 + 64 * 64 + 16 * 64) * 2;
constexpr int kMlpParams = 64 * 15 + 64 + 64 * 64 + 64 + 3 * 64 + 3;   // float32 master parameters

struct MlpDev {
    const uint16_t* wtiles;   // kMlpWeightBytes
    const float* bias;        // b1[64], b2[64], b3[16] (zero padded)
    float in_mean[16], in_inv_std[16];
    float out_mean[4], out_std[4];
};

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B (both
// K-major), FP32 accumulator, M x N tile.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Offsets of the parameter blocks in the float32 master / gradient vectors.
constexpr int kGradW1 = 0;
constexpr int kGradB1 = kGradW1 + 64 * 15;
constexpr int kGradW2 = kGradB1 + 64;
constexpr int kGradB2 = kGradW2 + 64 * 64;
constexpr int kGradW3 = kGradB2 + 64;
constexpr int kGradB3 = kGradW3 + 3 * 64;

struct TrainDev {
    const uint16_t* wtiles;   // W1 | W2 | W3 BF16 tiles (forward)
    const uint16_t* btiles;   // W3^T (64 x 16) | W2^T (64 x 64) BF16 tiles (backward)
    const float* bias;        // 144
    float in_mean[16], in_inv_std[16];
    float out_mean[4], out_inv_std[4];
    float grad_scale;         // 2 / (3 * sum of row weights): gradient of the weighted mean squared error
    float* grad;              // [kMlpParams] float32 accumulators
    float* loss;              // [1] sum over rows of w * |y - t|^2 (normalised units)
};

size_t mlp_forward_smem_bytes();
size_t mlp_train_smem_bytes();

// Accumulates the loss gradient of a batch into P.grad and its weighted sum
// of squared errors into P.loss (targ [rows][4] raw targets, wrow [rows] row weights).
cudaError_t launch_mlp_train(const TrainDev& P, const float4* feat, const float4* targ, const float* wrow,
                             long long rows, int* err, int n_sm, cudaStream_t st);
cudaError_t launch_mlp_pack(const float* master, uint16_t* wtiles, uint16_t* btiles, float* bias, cudaStream_t st);
cudaError_t launch_adam(float* master, float* m, float* v, float* grad, int n, float lr, int t, cudaStream_t st);

// Frozen normalisation of a training batch (rows of positive weight):
// norm[36] float32 = in_mean[15], in_std[15], out_mean[3], out_std[3]; acc is
// device scratch of 38 doubles; acc[18] holds the row count afterwards.
cudaError_t launch_norm_stats(const float4* feat, const float4* targ, const float* wrow, long long rows, double* acc,
                              float* norm, int n_sm, cudaStream_t st);

// out[r] = (de-normalised network output of feat[r], 0); feat is [rows][16]
// raw features (the 16th ignored); err gets bit 0 on an MMA timeout.
cudaError_t launch_mlp_forward(const MlpDev& net, const float4* feat, float4* out, long long rows, int* err,
                               int n_sm, cudaStream_t st);

// Packs float32 master parameters (W1[64][15], b1, W2[64][64], b2, W3[3][64],
// b3) into BF16 tiles and the padded bias vector.
void pack_mlp_weights(const float* params, uint16_t* tiles, float* bias);

}  // namespace ffsrl
