// Host-callable launchers of the XPBD kernels (internal to the library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "xpbd_device.cuh"

namespace ffsrl {

// Dynamic shared memory of one step CTA: positions (resident only), the
// two-stage constraint ring (ring only), the segment table and contact bits.
size_t step_smem_bytes(int Vp, bool resident, bool ring, int ring_bytes, int n_seg);

// Step kernel over n_blocks envs (env_list NULL: envs 0..n_blocks-1).
cudaError_t launch_step(const SimDev& S, bool resident, bool ring, int block, const int* env_list, int n_blocks,
                        size_t smem_bytes, cudaStream_t stream, const float* actions, float* obs,
                        float* reward, uint8_t* done);
cudaError_t launch_reset(const SimDev& S, const uint8_t* mask, unsigned long long seed, cudaStream_t st);
cudaError_t launch_pack(const SimDev& S, const int* pstart, float* x, float* v, cudaStream_t st);
cudaError_t launch_unpack(const SimDev& S, const int* pstart, const float* x, const float* v, cudaStream_t st);

}  // namespace ffsrl
