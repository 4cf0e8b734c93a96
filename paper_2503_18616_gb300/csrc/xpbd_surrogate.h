// Surrogate-assisted substep kernels (internal to the library).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mlp_tc.h"
#include "xpbd_device.cuh"

namespace ffsrl {

constexpr int kSubstepSurrogate = 1;  // add the network's correction, 1 iteration, residual check, fallback
constexpr int kSubstepRecord = 2;     // full solve, write training targets

struct SubstepCtl {
    int mode;
    int last;               // last substep of the step: contacts, observation, reward, done
    const float4* dx;       // [stride] network corrections (surrogate mode)
    float4* target;         // [stride] solve minus prediction (record mode; may be null)
    float threshold;        // residual above which the surrogate substep falls back
    int check;              // evaluate the residual (a finite threshold, or a residual output)
    int decide;             // fall back unless residual <= threshold (a finite threshold; +inf never falls back)
    int n_full;             // iterations of the full solve
    float* lambda;          // multipliers of the full solve (per env at EnvDev::loff)
    int* fallbacks;         // [n_env] counters (may be null)
    float* residual;        // [n_env] running max of the checked residual (may be null)
    float4* scratch;        // [stride] corrections of the fused step (slot order per env)
    float4* vpred;          // [stride] predicted velocities of the fused step (slot order per env)
    uint4* arows;           // [2 (stride + 128 n_env)] network input tiles of the fused step
};

size_t substep_smem_bytes(int Vp, bool resident);

cudaError_t launch_features(const SimDev& S, const int* env_list, int n_list, bool update_tool,
                            const float* actions, float4* F, cudaStream_t st);
cudaError_t launch_substep(const SimDev& S, const SubstepCtl& C, const int* env_list, int n_list, bool resident,
                           size_t smem, cudaStream_t st, float* obs, float* reward, uint8_t* done);

// Fused warm-start step: every substep of the step in one launch, one CTA of
// kWarmThreads threads per env with the env resident in shared memory (the
// network on the tensor cores inside the same CTA). C.scratch and C.vpred hold
// [stride] float4 each, C.arows 32 bytes per row plus 4 KB per env (env e's
// tiles start at row voff_e + 128 e); C.mode, C.last, C.dx and C.target are
// ignored.
constexpr int kWarmThreads = 256;
constexpr int kWarmMaxDegree = 23;   // 1-ring size the fused kernel gathers (a 48-byte record per slot)
// jit: the kernel that builds each tile's input just in time and keeps the
// network outputs in TMEM until applied (meshes with tile_reach <= 4; it does
// not use C.scratch or C.arows); else the kernel that stages both in global
// memory.
constexpr int kWarmJitMaxReach = 4;
size_t warm_smem_bytes(int Vp, int ring_bytes, int n_seg, bool jit);
cudaError_t configure_warm_step(size_t smem, bool jit);   // shared-memory limit, ahead of stream capture
cudaError_t launch_warm_step(const SimDev& S, const MlpDev& net, const SubstepCtl& C, const int* env_list,
                             int n_list, size_t smem, bool jit, const float* actions, float* obs, float* reward,
                             uint8_t* done, cudaStream_t st);

}  // namespace ffsrl
