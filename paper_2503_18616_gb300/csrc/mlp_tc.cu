// Per-vertex warm-start network on the 5th-generation tensor cores (sm_103a).
//
// The network (not in the FF-SRL paper; the learned warm-start of the
// workload) maps 15 features of a vertex to a 3-vector correction:
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

namespace ffsrl {

namespace {

__device__ __forceinline__ uint32_t saddr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor of a K-major operand without swizzling.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = uint64_t((addr & 0x3FFFFu) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;  // descriptor version of the 5th-generation tensor cores
    return d;                // base offset 0, relative leading offset, no swizzle
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Round-to-nearest-even BF16 bits of a float (finite inputs).
__device__ __forceinline__ uint32_t bf16_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

// Byte offset of the 16-byte chunk (row r, k-chunk kc) in a K-major tile with kcs chunks per row.
__device__ __forceinline__ uint32_t tile_off(int r, int kc, int kcs) {
    return uint32_t(((r >> 3) * kcs + kc) * 128 + (r & 7) * 16);
}

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
