// On-chip peak probes (include/ffsrl_probe.h): FP32 FMA throughput and
// shared-memory load bandwidth of the current device, timed with CUDA events.
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/ffsrl.h"
#include "../../include/ffsrl_probe.h"

namespace ffsrl {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kThreads = 1024;
constexpr int kCtasPerSm = 2;
constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kUnroll = 16;    // FMAs per chain per loop trip
constexpr int kWords = 2048;   // 16-byte words in the shared-memory buffer (32 KB)
constexpr int kLoads = 8;      // loads per thread per loop trip

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = float(threadIdx.x) * 1e-7f + float(c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.f) out[blockIdx.x] = s;   // never true (x stays positive); keeps the chains live
}

__global__ void __launch_bounds__(kThreads) smem_probe_kernel(unsigned* out, int iters) {
    __shared__ uint4 buf[kWords];
    for (int i = threadIdx.x; i < kWords; i += blockDim.x) buf[i] = make_uint4(i, 3u * i, 5u * i, 7u * i);
    __syncthreads();
    unsigned a0 = 0u, a1 = 0u;
    const int t = int(threadIdx.x);
    for (int it = 0; it < iters; ++it) {
        // a quarter warp reads 8 consecutive words from a multiple of 8: one
        // whole 128-byte line, every bank once. The kLoads words of a thread
        // are distinct (offsets u x 256 below the 2048-word buffer), so none
        // of the loads repeats another, and the start moves every trip.
#pragma unroll
        for (int u = 0; u < kLoads; ++u) {
            const uint4 v = buf[(t + u * (kWords / kLoads) + it * 32) & (kWords - 1)];
            a0 ^= v.x ^ v.y;
            a1 ^= v.z ^ v.w;
        }
    }
    if ((a0 ^ a1) == 0x9e3779b9u) out[blockIdx.x] = a0;   // keeps the loads live
}

template <class K>
int time_launches(K launch, int repeats, double* best_ms) {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e30;
    if (e == cudaSuccess) e = launch(st);   // warm-up
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch(st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        ffsrl::set_last_error(std::string("peak probe: ") + cudaGetErrorString(e));
        return FFSRL_E_CUDA;
    }
    *best_ms = best;
    return FFSRL_OK;
}

int n_sms(int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        ffsrl::set_last_error(std::string("peak probe: ") + cudaGetErrorString(e));
        return FFSRL_E_CUDA;
    }
    return FFSRL_OK;
}

}  // namespace

extern "C" int ffsrl_probe_fp32(int32_t repeats, double* tflops, double* ms) {
    if (repeats < 1 || !tflops || !ms) {
        ffsrl::set_last_error("ffsrl_probe_fp32: need repeats >= 1 and output pointers");
        return FFSRL_E_INVAL;
    }
    int sms = 0;
    int rc = n_sms(&sms);
    if (rc) return rc;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * size_t(sms) * kCtasPerSm) != cudaSuccess) {
        ffsrl::set_last_error("ffsrl_probe_fp32: cudaMalloc failed");
        return FFSRL_E_CUDA;
    }
    const int grid = sms * kCtasPerSm, iters = 20000;
    double best = 0;
    rc = time_launches(
        [&](cudaStream_t st) {
            fma_probe_kernel<<<grid, kThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
            return cudaGetLastError();
        },
        repeats, &best);
    cudaFree(out);
    if (rc) return rc;
    const double fmas = double(grid) * kThreads * double(iters) * kUnroll * kChains;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    *ms = best;
    return FFSRL_OK;
}

extern "C" int ffsrl_probe_smem(int32_t repeats, double* gbs, double* ms) {
    if (repeats < 1 || !gbs || !ms) {
        ffsrl::set_last_error("ffsrl_probe_smem: need repeats >= 1 and output pointers");
        return FFSRL_E_INVAL;
    }
    int sms = 0;
    int rc = n_sms(&sms);
    if (rc) return rc;
    unsigned* out = nullptr;
    if (cudaMalloc(&out, sizeof(unsigned) * size_t(sms) * kCtasPerSm) != cudaSuccess) {
        ffsrl::set_last_error("ffsrl_probe_smem: cudaMalloc failed");
        return FFSRL_E_CUDA;
    }
    const int grid = sms * kCtasPerSm, iters = 20000;
    double best = 0;
    rc = time_launches(
        [&](cudaStream_t st) {
            smem_probe_kernel<<<grid, kThreads, 0, st>>>(out, iters);
            return cudaGetLastError();
        },
        repeats, &best);
    cudaFree(out);
    if (rc) return rc;
    const double bytes = double(grid) * kThreads * double(iters) * kLoads * 16.0;
    *gbs = bytes / (best * 1e-3) / 1e9;
    *ms = best;
    return FFSRL_OK;
}
