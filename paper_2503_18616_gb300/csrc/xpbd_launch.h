// Host-callable launchers of the XPBD kernels (internal to the library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "xpbd_device.cuh"

namespace ffsrl {

// Execution schedule of one step-kernel launch.
struct StepConfig {
    int sub = 256;        // threads per env
    int envs = 1;         // envs per CTA (sharing one constraint ring)
    bool resident = true; // positions in shared memory
    bool ring = true;     // constraint records through the TMA double buffer
    int occ = 0;          // CTAs per SM the registers are budgeted for (0: the block size's default)
};

// Dynamic shared memory of one step CTA: positions of its envs (resident
// only), the two-stage constraint ring (ring only), the segment table and
// contact bits.
size_t step_smem_bytes(int Vp, bool resident, bool ring, int ring_bytes, int n_seg, int envs);

// Whether a (sub, envs, resident, ring, occ) combination is compiled.
bool step_config_supported(int sub, int envs, bool resident, bool ring, int occ = 0);

// Step kernel over the n_list envs of env_list (NULL: envs 0..n_list-1), all of one mesh.
cudaError_t launch_step(const SimDev& S, const StepConfig& c, const int* env_list, int n_list,
                        size_t smem_bytes, cudaStream_t stream, const float* actions, float* obs,
                        float* reward, uint8_t* done);
// Sets the kernel's dynamic shared-memory limit for a launch of this size
// (done by launch_step too; called ahead of stream capture).
cudaError_t configure_step(const StepConfig& c, size_t smem_bytes);
// CTAs of this configuration that fit one SM with smem_bytes of dynamic shared memory.
int step_max_active(const StepConfig& c, size_t smem_bytes);
// CTAs per SM the configuration's registers are budgeted for.
int step_ctas_per_sm(const StepConfig& c);
// Cluster step (xpbd_cluster.cu): envs whose mesh variant has parts = cl
// ranges, sub threads per CTA, cl CTAs per env; smem from cluster_smem_bytes.
constexpr int kClusterThreads = 1024;   // threads per CTA of the cluster kernel
size_t cluster_smem_bytes(int part_slots);
bool cluster_config_supported(int sub, int cl);
cudaError_t launch_cluster_step(const SimDev& S, int sub, int cl, const int* env_list, int n_list, size_t smem,
                                cudaStream_t st, const float* actions, float* obs, float* reward, uint8_t* done);
// Clusters of this shape that fit on the device at once (0: cannot launch);
// also sets the kernel's shared-memory limit.
int cluster_max_active(int sub, int cl, size_t smem);

// Jacobi step (xpbd_jacobi.cu): one CTA of 256 threads per env, positions and
// the per-vertex correction sums in shared memory.
size_t jacobi_smem_bytes(int Vp);
cudaError_t configure_jacobi_step(size_t smem);
cudaError_t launch_jacobi_step(const SimDev& S, const int* env_list, int n_list, size_t smem, cudaStream_t st,
                               const float* actions, float* obs, float* reward, uint8_t* done);

cudaError_t launch_reset(const SimDev& S, const uint8_t* mask, unsigned long long seed, cudaStream_t st);
cudaError_t launch_auto_reset(const SimDev& S, cudaStream_t st);
cudaError_t launch_set_clamp(const SimDev& S, const float* angles, cudaStream_t st);
cudaError_t launch_pack(const SimDev& S, const int* pstart, float* x, float* v, cudaStream_t st);
cudaError_t launch_unpack(const SimDev& S, const int* pstart, const float* x, const float* v, cudaStream_t st);

}  // namespace ffsrl
