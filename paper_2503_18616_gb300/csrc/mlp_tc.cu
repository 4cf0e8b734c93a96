// Per-vertex warm-start network on the 5th-generation tensor cores (sm_103a).
//
// The network (not in the FF-SRL paper; a learned warm-start added to the
// method) maps 15 features of a vertex to a 3-vector correction:
// 15 -> 64 -> ReLU -> 64 -> ReLU -> 3, BF16 weights and activations, FP32
// accumulation. One CTA of 128 threads processes 128-row tiles: each row is
// one TMEM lane and one thread of the epilogue.
//
// Per tile: the threads normalise their row's features, round them to BF16
// and store them as the A operand (128 x 16) in shared memory; one elected
// thread issues tcgen05.mma (M = 128, K = 16 per instruction) against the
// weight tiles staged once per CTA, the accumulators land in TMEM, and the
// epilogue reads them back with tcgen05.ld, adds the bias, applies ReLU,
// rounds to BF16 and stores the next layer's A operand. Completion of each
// MMA chain is tracked by tcgen05.commit on an mbarrier; waits are bounded
// and a timeout is reported through the error flag.
//
// Operand layout (both A and B K-major, no swizzle): an R x K BF16 tile is a
// grid of 8 x 8 "core matrices" (8 rows of 16 bytes, stored contiguously);
// core matrix (r / 8, k / 8) lives at byte ((r / 8) * (K / 8) + k / 8) * 128.
// The descriptor's leading-dimension offset is therefore 128 bytes (next core
// matrix along K) and the stride-dimension offset (K / 8) * 128 bytes (next
// group of 8 rows).
#include <cstdint>
#include <cstring>

#include "mlp_tc.h"
#include "tc_prims.cuh"

namespace ffsrl {

using namespace tc;

namespace {

constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 128;

}  // namespace

__global__ void __launch_bounds__(128) mlp_forward_kernel(MlpDev net, const float4* __restrict__ feat,
                                                          float4* __restrict__ out, long long rows,
                                                          int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char* Wt = sm;                        // W1 (64x16) | W2 (64x64) | W3 (16x64)
    unsigned char* At = sm + kMlpWeightBytes;      // 128 x 16 input tile
    unsigned char* Ht = At + 4096;                 // 128 x 64 hidden tile
    float* bias = reinterpret_cast<float*>(Ht + 16384);   // b1[64] b2[64] b3[16]
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < kMlpWeightBytes / 16; i += 128)
        reinterpret_cast<uint4*>(Wt)[i] = reinterpret_cast<const uint4*>(net.wtiles)[i];
    for (int i = tid; i < 144; i += 128) bias[i] = net.bias[i];
    if (tid == 0) mbar_init(&mbar);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lane_base = uint32_t(32 * warp) << 16;   // this warp's TMEM lanes
    const uint32_t idesc64 = umma_idesc_bf16(128, 64), idesc16 = umma_idesc_bf16(128, 16);
    const uint32_t aW1 = saddr(Wt), aW2 = aW1 + 2048, aW3 = aW1 + 10240, aA = saddr(At), aH = saddr(Ht);
    uint32_t phase = 0;
    bool ok = true, failed = false;

    for (long long tile = blockIdx.x; tile * kRows < rows; tile += gridDim.x) {
        const long long row = tile * kRows + tid;
        const bool valid = row < rows;
        // Stage the normalised BF16 input row (feature 16 is padding).
        {
            float f[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = valid ? feat[row * 4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
                f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
            }
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float a = 2 * k < 15 ? (f[2 * k] - net.in_mean[2 * k]) * net.in_inv_std[2 * k] : 0.f;
                const float b = 2 * k + 1 < 15 ? (f[2 * k + 1] - net.in_mean[2 * k + 1]) * net.in_inv_std[2 * k + 1] : 0.f;
                p[k] = bf16_bits(valid ? a : 0.f) | (bf16_bits(valid ? b : 0.f) << 16);
            }
            *reinterpret_cast<uint4*>(At + tile_off(tid, 0, 2)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(At + tile_off(tid, 1, 2)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        // Layer 1: D[0:64) = A (128x16) W1^T.
        if (tid == 0) {
            umma_bf16(tmem, umma_desc(aA, 128, 256), umma_desc(aW1, 128, 256), idesc64, 0);
            umma_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase & 1);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        ++phase;
        fence_after_sync();
        // Epilogue 1: bias, ReLU, BF16 -> hidden tile.
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + c0, v);
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                p[k] = bf16_bits(fmaxf(v[2 * k] + bias[c0 + 2 * k], 0.f)) |
                       (bf16_bits(fmaxf(v[2 * k + 1] + bias[c0 + 2 * k + 1], 0.f)) << 16);
            *reinterpret_cast<uint4*>(Ht + tile_off(tid, c0 / 8, 8)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(Ht + tile_off(tid, c0 / 8 + 1, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        // Layer 2: D[64:128) = H1 (128x64) W2^T, four K = 16 steps.
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                umma_bf16(tmem + 64, umma_desc(aH + 256 * j, 128, 1024), umma_desc(aW2 + 256 * j, 128, 1024), idesc64,
                          j);
            umma_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase & 1);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        ++phase;
        fence_after_sync();
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + 64 + c0, v);
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                p[k] = bf16_bits(fmaxf(v[2 * k] + bias[64 + c0 + 2 * k], 0.f)) |
                       (bf16_bits(fmaxf(v[2 * k + 1] + bias[64 + c0 + 2 * k + 1], 0.f)) << 16);
            *reinterpret_cast<uint4*>(Ht + tile_off(tid, c0 / 8, 8)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(Ht + tile_off(tid, c0 / 8 + 1, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        // Layer 3: D[0:16) = H2 (128x64) W3^T (rows 3..15 of W3 are zero).
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                umma_bf16(tmem, umma_desc(aH + 256 * j, 128, 1024), umma_desc(aW3 + 256 * j, 128, 1024), idesc16, j);
            umma_commit(&mbar);
        }
        ok = mbar_wait(&mbar, phase & 1);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        ++phase;
        fence_after_sync();
        {
            float v[16];
            tmem_ld16(tmem + lane_base, v);
            if (valid) {
                const float y0 = (v[0] + bias[128]) * net.out_std[0] + net.out_mean[0];
                const float y1 = (v[1] + bias[129]) * net.out_std[1] + net.out_mean[1];
                const float y2 = (v[2] + bias[130]) * net.out_std[2] + net.out_mean[2];
                out[row] = make_float4(y0, y1, y2, 0.f);
            }
        }
        fence_before_sync();
        __syncthreads();   // the next tile overwrites the input tile and TMEM columns 0..63
        fence_after_sync();
    }
    if (failed) {
        // An MMA chain did not signal completion: wait once more (bounded)
        // for the commit in flight before freeing TMEM, then report.
        mbar_wait(&mbar, phase & 1);
        if (tid == 0) atomicOr(err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

size_t mlp_forward_smem_bytes() {
    // Operand tiles and biases need 33 KB; the allocation is padded to 64 KB
    // so that at most three CTAs (3 x 128 TMEM columns of 512) share an SM.
    return 64 * 1024;
}

cudaError_t launch_mlp_forward(const MlpDev& net, const float4* feat, float4* out, long long rows, int* err,
                               int n_sm, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(mlp_forward_smem_bytes()));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long long tiles = (rows + kRows - 1) / kRows;
    const int grid = int(tiles < 3LL * n_sm ? tiles : 3LL * n_sm);
    mlp_forward_kernel<<<grid, 128, mlp_forward_smem_bytes(), st>>>(net, feat, out, rows, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Training: fused forward + backward per 128-row tile on the tensor cores.
//
// Per tile (thread = row = TMEM lane): forward as above, keeping the ReLU
// masks of both hidden layers; the loss gradient dY = scale * w * (y - t) of
// the normalised output; then
//   dH2 = dY W3   (MMA, B = W3^T tile)   -> dZ2 = dH2 * [H2 > 0]
//   dH1 = dZ2 W2  (MMA, B = W2^T tile)   -> dZ1 = dH1 * [H1 > 0]
// and the weight gradients as two more MMAs whose K dimension is the tile's
// 128 rows, accumulated in TMEM over all tiles of the CTA:
//   [dZ2^T ; dZ1^T] (128 x 128) [H1 | X] (80 x 128)^T -> dW2 (rows 0..63,
//   cols 0..63) and dW1 (rows 64..127, cols 64..79)
//   [dY^T ; 0] (128 x 128) H2 (64 x 128)^T            -> dW3 (rows 0..2)
// The transposed operand tiles are written by the epilogue threads. Bias
// gradients and the loss are reduced with warp shuffles. At the end each CTA
// adds its gradients to the global FP32 accumulators.
// ---------------------------------------------------------------------------

namespace {

// 2-byte element (row n, column k) of a K-major tile with kcs chunks per row.
__device__ __forceinline__ void st_elem(unsigned char* tile, int n, int k, int kcs, uint32_t bits16) {
    *reinterpret_cast<uint16_t*>(tile + ((n >> 3) * kcs + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2) =
        uint16_t(bits16);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Offsets of the smem regions of the training kernel.
constexpr int kTrW = 0;                       // W1 | W2 | W3       12288
constexpr int kTrB = kTrW + kMlpWeightBytes;  // W3T | W2T          10240
constexpr int kTrX = kTrB + 10240;            // X (128 x 16)        4096
constexpr int kTrH1 = kTrX + 4096;            // H1, later dZ2      16384
constexpr int kTrH2 = kTrH1 + 16384;          // H2                 16384
constexpr int kTrDY = kTrH2 + 16384;          // dY (128 x 16)       4096
constexpr int kTrAW = kTrDY + 4096;           // [dZ2^T; dZ1^T]     32768
constexpr int kTrBW = kTrAW + 32768;          // [H1^T; X^T]        20480
constexpr int kTrAY = kTrBW + 20480;          // [dY^T; 0]          32768
constexpr int kTrBH = kTrAY + 32768;          // H2^T               16384
constexpr int kTrRed = kTrBH + 16384;         // db1, db2, db3, loss   4 * 136
constexpr int kTrBias = kTrRed + 4 * 136;     // b1, b2, b3            4 * 144
constexpr int kTrSmem = kTrBias + 4 * 144;

constexpr uint32_t kTrTmemCols = 512;

}  // namespace

__global__ void __launch_bounds__(128) mlp_train_kernel(TrainDev P, const float4* __restrict__ feat,
                                                        const float4* __restrict__ targ,
                                                        const float* __restrict__ wrow, long long rows,
                                                        int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* red = reinterpret_cast<float*>(sm + kTrRed);   // db1[64] db2[64] db3[4] loss[1]
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kTrTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < kMlpWeightBytes / 16; i += 128)
        reinterpret_cast<uint4*>(sm + kTrW)[i] = reinterpret_cast<const uint4*>(P.wtiles)[i];
    for (int i = tid; i < 10240 / 16; i += 128)
        reinterpret_cast<uint4*>(sm + kTrB)[i] = reinterpret_cast<const uint4*>(P.btiles)[i];
    for (int i = tid; i < 32768 / 16; i += 128) reinterpret_cast<uint4*>(sm + kTrAY)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 136; i += 128) red[i] = 0.f;
    float* bias = reinterpret_cast<float*>(sm + kTrBias);
    for (int i = tid; i < 144; i += 128) bias[i] = P.bias[i];
    if (tid == 0) mbar_init(&mbar);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lb = uint32_t(32 * warp) << 16;
    const uint32_t aW1 = saddr(sm + kTrW), aW2 = aW1 + 2048, aW3 = aW1 + 10240;
    const uint32_t aW3T = saddr(sm + kTrB), aW2T = aW3T + 2048;
    const uint32_t aX = saddr(sm + kTrX), aH1 = saddr(sm + kTrH1), aH2 = saddr(sm + kTrH2), aDY = saddr(sm + kTrDY);
    const uint32_t aAW = saddr(sm + kTrAW), aBW = saddr(sm + kTrBW), aAY = saddr(sm + kTrAY), aBH = saddr(sm + kTrBH);
    unsigned char* X = sm + kTrX;
    unsigned char* H1 = sm + kTrH1;
    unsigned char* H2 = sm + kTrH2;
    unsigned char* DY = sm + kTrDY;
    unsigned char* AW = sm + kTrAW;
    unsigned char* BW = sm + kTrBW;
    unsigned char* AY = sm + kTrAY;
    unsigned char* BH = sm + kTrBH;
    uint32_t phase = 0;
    bool failed = false;
    int n_tiles = 0;
    const int r = tid;

    auto sync_for_mma = [&]() {
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    };
    auto wait_mma = [&]() -> bool {
        const bool ok = mbar_wait(&mbar, phase & 1);
        if (__syncthreads_or(!ok)) return false;
        ++phase;
        fence_after_sync();
        return true;
    };

    for (long long tile = blockIdx.x; tile * 128 < rows; tile += gridDim.x) {
        const long long row = tile * 128 + r;
        const bool valid = row < rows;
        const float w = valid ? wrow[row] : 0.f;
        // -- stage X (normalised, BF16) and X^T --------------------------------
        {
            float f[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = valid ? feat[row * 4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
                f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
            }
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float a = (valid && k < 15) ? (f[k] - P.in_mean[k]) * P.in_inv_std[k] : 0.f;
                const float b = (valid && k + 1 < 15) ? (f[k + 1] - P.in_mean[k + 1]) * P.in_inv_std[k + 1] : 0.f;
                const uint32_t ba = bf16_bits(a), bb = bf16_bits(b);
                p[k / 2] = ba | (bb << 16);
                st_elem(BW, 64 + k, r, 16, ba);
                st_elem(BW, 64 + k + 1, r, 16, bb);
            }
            *reinterpret_cast<uint4*>(X + tile_off(r, 0, 2)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(X + tile_off(r, 1, 2)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        sync_for_mma();
        if (tid == 0) {
            umma_bf16(tmem, umma_desc(aX, 128, 256), umma_desc(aW1, 128, 256), umma_idesc_bf16(128, 64), 0);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        // -- H1 = relu(D1 + b1): tile, H1^T, mask ------------------------------
        uint64_t m1 = 0, m2 = 0;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + c0, v);
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float a = fmaxf(v[k] + bias[c0 + k], 0.f), b = fmaxf(v[k + 1] + bias[c0 + k + 1], 0.f);
                m1 |= uint64_t(a > 0.f) << (c0 + k);
                m1 |= uint64_t(b > 0.f) << (c0 + k + 1);
                const uint32_t ba = bf16_bits(a), bb = bf16_bits(b);
                p[k / 2] = ba | (bb << 16);
                st_elem(BW, c0 + k, r, 16, ba);
                st_elem(BW, c0 + k + 1, r, 16, bb);
            }
            *reinterpret_cast<uint4*>(H1 + tile_off(r, c0 / 8, 8)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(H1 + tile_off(r, c0 / 8 + 1, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                umma_bf16(tmem + 64, umma_desc(aH1 + 256 * j, 128, 1024), umma_desc(aW2 + 256 * j, 128, 1024),
                          umma_idesc_bf16(128, 64), j);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        // -- H2 = relu(D2 + b2): tile, H2^T, mask ------------------------------
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + 64 + c0, v);
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float a = fmaxf(v[k] + bias[64 + c0 + k], 0.f), b = fmaxf(v[k + 1] + bias[64 + c0 + k + 1], 0.f);
                m2 |= uint64_t(a > 0.f) << (c0 + k);
                m2 |= uint64_t(b > 0.f) << (c0 + k + 1);
                const uint32_t ba = bf16_bits(a), bb = bf16_bits(b);
                p[k / 2] = ba | (bb << 16);
                st_elem(BH, c0 + k, r, 16, ba);
                st_elem(BH, c0 + k + 1, r, 16, bb);
            }
            *reinterpret_cast<uint4*>(H2 + tile_off(r, c0 / 8, 8)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(H2 + tile_off(r, c0 / 8 + 1, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                umma_bf16(tmem, umma_desc(aH2 + 256 * j, 128, 1024), umma_desc(aW3 + 256 * j, 128, 1024),
                          umma_idesc_bf16(128, 16), j);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        // -- loss gradient dY (normalised output units) -------------------------
        float g[3];
        {
            float v[16];
            tmem_ld16(tmem + lb, v);
            const float4 t4 = valid ? targ[row] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float tt[3] = {t4.x, t4.y, t4.z};
            float l = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float y = v[k] + bias[128 + k];
                const float d = y - (tt[k] - P.out_mean[k]) * P.out_inv_std[k];
                l += w * d * d;
                g[k] = P.grad_scale * w * d;
            }
            const uint32_t g0 = bf16_bits(g[0]), g1 = bf16_bits(g[1]), g2 = bf16_bits(g[2]);
            *reinterpret_cast<uint4*>(DY + tile_off(r, 0, 2)) = make_uint4(g0 | (g1 << 16), g2, 0u, 0u);
            *reinterpret_cast<uint4*>(DY + tile_off(r, 1, 2)) = make_uint4(0u, 0u, 0u, 0u);
            st_elem(AY, 0, r, 16, g0);
            st_elem(AY, 1, r, 16, g1);
            st_elem(AY, 2, r, 16, g2);
            l = warp_sum(l);
            if (lane == 0) atomicAdd(&red[132], l);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float s = warp_sum(g[k]);
                if (lane == 0) atomicAdd(&red[128 + k], s);
            }
        }
        sync_for_mma();
        if (tid == 0) {
            umma_bf16(tmem, umma_desc(aDY, 128, 256), umma_desc(aW3T, 128, 256), umma_idesc_bf16(128, 64), 0);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        // -- dZ2 = dH2 * [H2 > 0]: tile (into H1's space), dZ2^T, db2 -----------
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + c0, v);
            uint32_t p[8];
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float a = ((m2 >> (c0 + k)) & 1) ? v[k] : 0.f;
                const float b = ((m2 >> (c0 + k + 1)) & 1) ? v[k + 1] : 0.f;
                const uint32_t ba = bf16_bits(a), bb = bf16_bits(b);
                p[k / 2] = ba | (bb << 16);
                st_elem(AW, c0 + k, r, 16, ba);
                st_elem(AW, c0 + k + 1, r, 16, bb);
                const float sa = warp_sum(a), sb = warp_sum(b);
                if (lane == 0) {
                    atomicAdd(&red[64 + c0 + k], sa);
                    atomicAdd(&red[64 + c0 + k + 1], sb);
                }
            }
            *reinterpret_cast<uint4*>(H1 + tile_off(r, c0 / 8, 8)) = make_uint4(p[0], p[1], p[2], p[3]);
            *reinterpret_cast<uint4*>(H1 + tile_off(r, c0 / 8 + 1, 8)) = make_uint4(p[4], p[5], p[6], p[7]);
        }
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                umma_bf16(tmem + 64, umma_desc(aH1 + 256 * j, 128, 1024), umma_desc(aW2T + 256 * j, 128, 1024),
                          umma_idesc_bf16(128, 64), j);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        // -- dZ1 = dH1 * [H1 > 0]: dZ1^T, db1 ------------------------------------
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + 64 + c0, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = ((m1 >> (c0 + k)) & 1) ? v[k] : 0.f;
                st_elem(AW, 64 + c0 + k, r, 16, bf16_bits(a));
                const float sa = warp_sum(a);
                if (lane == 0) atomicAdd(&red[c0 + k], sa);
            }
        }
        sync_for_mma();
        // -- weight gradients, accumulated in TMEM across tiles -----------------
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                umma_bf16(tmem + 128, umma_desc(aAW + 256 * j, 128, 2048), umma_desc(aBW + 256 * j, 128, 2048),
                          umma_idesc_bf16(128, 80), (n_tiles > 0 || j > 0) ? 1 : 0);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                umma_bf16(tmem + 256, umma_desc(aAY + 256 * j, 128, 2048), umma_desc(aBH + 256 * j, 128, 2048),
                          umma_idesc_bf16(128, 64), (n_tiles > 0 || j > 0) ? 1 : 0);
            umma_commit(&mbar);
        }
        if (!wait_mma()) { failed = true; break; }
        ++n_tiles;
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
    }
    if (failed) {
        mbar_wait(&mbar, phase & 1);
        if (tid == 0) atomicOr(err, 1);
    } else if (n_tiles > 0) {
        // Add this CTA's gradients to the global accumulators.
        float* G = P.grad;
        for (int c0 = 0; c0 < 80; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + 128 + c0, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int n = c0 + k;
                if (r < 64 && n < 64) atomicAdd(&G[kGradW2 + r * 64 + n], v[k]);
                if (r >= 64 && n >= 64 && n < 79) atomicAdd(&G[kGradW1 + (r - 64) * 15 + (n - 64)], v[k]);
            }
        }
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lb + 256 + c0, v);
            if (r < 3)
#pragma unroll
                for (int k = 0; k < 16; ++k) atomicAdd(&G[kGradW3 + r * 64 + c0 + k], v[k]);
        }
        __syncthreads();
        if (tid < 64) {
            atomicAdd(&G[kGradB1 + tid], red[tid]);
            atomicAdd(&G[kGradB2 + tid], red[64 + tid]);
        }
        if (tid < 3) atomicAdd(&G[kGradB3 + tid], red[128 + tid]);
        if (tid == 0) atomicAdd(P.loss, red[132]);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTrTmemCols) : "memory");
}

// Repacks the float32 master parameters into the BF16 tiles of the forward
// (W1, W2, W3) and backward (W3^T, W2^T) passes and the padded biases.
__global__ void mlp_pack_kernel(const float* __restrict__ master, uint16_t* __restrict__ wtiles,
                                uint16_t* __restrict__ btiles, float* __restrict__ bias) {
    auto put = [](uint16_t* tile, int R, int K, int r, int k, float v) {
        const int off = ((r / 8) * (K / 8) + k / 8) * 64 + (r % 8) * 8 + (k % 8);
        const uint32_t u = __float_as_uint(v);
        tile[off] = uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
        (void)R;
    };
    const float* W1 = master + kGradW1;
    const float* W2 = master + kGradW2;
    const float* W3 = master + kGradW3;
    for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
        const int r = i / 16, k = i % 16;
        put(wtiles, 64, 16, r, k, k < 15 ? W1[r * 15 + k] : 0.f);
    }
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int r = i / 64, k = i % 64;
        put(wtiles + 1024, 64, 64, r, k, W2[r * 64 + k]);
        put(btiles + 1024, 64, 64, r, k, W2[k * 64 + r]);          // W2^T: row = input unit
    }
    for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) {
        const int r = i / 64, k = i % 64;
        put(wtiles + 1024 + 4096, 16, 64, r, k, r < 3 ? W3[r * 64 + k] : 0.f);
    }
    for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
        const int r = i / 16, k = i % 16;
        put(btiles, 64, 16, r, k, k < 3 ? W3[k * 64 + r] : 0.f);    // W3^T: row = hidden unit
    }
    for (int i = threadIdx.x; i < 144; i += blockDim.x)
        bias[i] = i < 64 ? master[kGradB1 + i] : i < 128 ? master[kGradB2 + i - 64] : i < 131 ? master[kGradB3 + i - 128] : 0.f;
}

// Adam (Kingma & Ba, ICLR 2015, Algorithm 1) on the float32 master
// parameters; clears the gradients afterwards.
__global__ void adam_kernel(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ grad, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        master[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        grad[i] = 0.f;
    }
}

// Frozen normalisation of the network's inputs and outputs (the warm-start's
// training data): column sums over the rows of positive weight, in double.
// Pass 0 sums the 15 features, the 3 targets and the row count into
// acc[0..18]; pass 1 sums the squared deviations from mean[0..17] into
// acc[19..36]. One atomic add per column and block.
constexpr int kNormCols = 18;

__global__ void __launch_bounds__(256) norm_stats_kernel(const float4* __restrict__ feat,
                                                         const float4* __restrict__ targ,
                                                         const float* __restrict__ wrow, long long rows, int pass,
                                                         double* __restrict__ acc) {
    __shared__ double s_part[8][kNormCols + 1];
    double sum[kNormCols + 1];
#pragma unroll
    for (int c = 0; c <= kNormCols; ++c) sum[c] = 0.0;
    double mean[kNormCols];
#pragma unroll
    for (int c = 0; c < kNormCols; ++c) mean[c] = pass ? acc[c] / acc[kNormCols] : 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
         r += (long long)gridDim.x * blockDim.x) {
        if (!(wrow[r] > 0.f)) continue;
        const float4* f = feat + 4 * r;
        const float4 a = f[0], b = f[1], c = f[2], d = f[3], t = targ[r];
        const float v[kNormCols] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z,
                                    t.x, t.y, t.z};
#pragma unroll
        for (int q = 0; q < kNormCols; ++q) {
            const double x = double(v[q]) - mean[q];
            sum[q] += pass ? x * x : x;
        }
        sum[kNormCols] += 1.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q <= kNormCols; ++q) {
        double x = sum[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_part[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x <= kNormCols && (pass == 0 || threadIdx.x < kNormCols)) {
        double x = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) x += s_part[w][threadIdx.x];
        if (x != 0.0) atomicAdd(&acc[(pass ? kNormCols + 1 : 0) + threadIdx.x], x);
    }
}

// norm[0..35] = in_mean[15], in_std[15], out_mean[3], out_std[3] (float32),
// population standard deviations, 1 for a column without spread.
__global__ void norm_finish_kernel(const double* __restrict__ acc, float* __restrict__ norm) {
    const int q = threadIdx.x;
    if (q >= kNormCols) return;
    const double n = acc[kNormCols];
    const double mean = acc[q] / n;
    const double sd = sqrt(acc[kNormCols + 1 + q] / n);
    const float s = sd > 0.0 ? float(sd) : 1.f;
    if (q < 15) {
        norm[q] = float(mean);
        norm[15 + q] = s;
    } else {
        norm[30 + q - 15] = float(mean);
        norm[33 + q - 15] = s;
    }
}

cudaError_t launch_norm_stats(const float4* feat, const float4* targ, const float* wrow, long long rows, double* acc,
                              float* norm, int n_sm, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * (kNormCols + 1) * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long long want = (rows + 255) / 256;
    const int grid = int(want < 4ll * n_sm ? (want > 0 ? want : 1) : 4ll * n_sm);
    for (int pass = 0; pass < 2; ++pass) {
        norm_stats_kernel<<<grid, 256, 0, st>>>(feat, targ, wrow, rows, pass, acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    norm_finish_kernel<<<1, 32, 0, st>>>(acc, norm);
    return cudaGetLastError();
}

size_t mlp_train_smem_bytes() { return size_t(kTrSmem); }

cudaError_t launch_mlp_train(const TrainDev& P, const float4* feat, const float4* targ, const float* wrow,
                             long long rows, int* err, int n_sm, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(mlp_train_smem_bytes()));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long long tiles = (rows + 127) / 128;
    const int grid = int(tiles < n_sm ? tiles : n_sm);   // one CTA per SM (512 TMEM columns each)
    mlp_train_kernel<<<grid, 128, mlp_train_smem_bytes(), st>>>(P, feat, targ, wrow, rows, err);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float* master, uint16_t* wtiles, uint16_t* btiles, float* bias, cudaStream_t st) {
    mlp_pack_kernel<<<1, 256, 0, st>>>(master, wtiles, btiles, bias);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* master, float* m, float* v, float* grad, int n, float lr, int t, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, float(t)), c2 = 1.f - powf(b2, float(t));
    adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(master, m, v, grad, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

// Host packing of the float32 master weights into BF16 K-major tiles.
static uint16_t host_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

static void pack_tile(const float* W, int out_rows, int in_cols, int R, int K, uint16_t* dst) {
    // W is [out_rows][in_cols] row-major; tile is R x K (zero padded).
    const int kcs = K / 8;
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const float v = (r < out_rows && k < in_cols) ? W[r * in_cols + k] : 0.f;
            const int off = ((r / 8) * kcs + k / 8) * 64 + (r % 8) * 8 + (k % 8);   // in uint16 units
            dst[off] = host_bf16(v);
        }
}

void pack_mlp_weights(const float* params, uint16_t* tiles, float* bias) {
    const float* W1 = params;
    const float* b1 = W1 + 64 * 15;
    const float* W2 = b1 + 64;
    const float* b2 = W2 + 64 * 64;
    const float* W3 = b2 + 64;
    const float* b3 = W3 + 3 * 64;
    pack_tile(W1, 64, 15, 64, 16, tiles);
    pack_tile(W2, 64, 64, 64, 64, tiles + 1024);
    pack_tile(W3, 3, 64, 16, 64, tiles + 1024 + 4096);
    for (int i = 0; i < 64; ++i) bias[i] = b1[i];
    for (int i = 0; i < 64; ++i) bias[64 + i] = b2[i];
    for (int i = 0; i < 16; ++i) bias[128 + i] = i < 3 ? b3[i] : 0.f;
}

}  // namespace ffsrl
