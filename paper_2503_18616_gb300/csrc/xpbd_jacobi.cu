// XPBD step with the paper's own parallel solver (Sec. III-A, sm_103a):
// Jacobi iterations in which every distance and volume constraint takes its
// step from the positions the iteration starts from, the corrections are
// summed per vertex (shared-memory atomics) and each vertex moves by its sum
// divided by the number of constraints that contain it. Multipliers are
// carried as in the Gauss-Seidel kernel. No colour order is needed: each
// iteration is one pass over the unpadded record lists (read from L2 with as
// many loads in flight as the loop allows) and two barriers, instead of one
// barrier per colour. The rest of the step (prediction, collision, velocity
// update, observation, reward) is that of the Gauss-Seidel kernel.
#include <cstdint>

#include "xpbd_device.cuh"
#include "xpbd_launch.h"
#include "xpbd_project.cuh"

namespace ffsrl {

namespace {

constexpr int kJacobiThreads = 256;

struct JacobiLayout {
    size_t x, acc, bits, total;
    __host__ __device__ explicit JacobiLayout(int Vp) {
        x = 0;
        acc = size_t(Vp) * 16;
        bits = acc + size_t(Vp) * 12;
        total = bits + size_t(Vp / 32) * 4;
    }
};

}  // namespace

size_t jacobi_smem_bytes(int Vp) { return JacobiLayout(Vp).total; }

__global__ void __launch_bounds__(kJacobiThreads, 3)
    xpbd_jacobi_kernel(SimDev S, const int* __restrict__ env_list, int n_list, const float* __restrict__ actions,
                       float* __restrict__ obs, float* __restrict__ reward, uint8_t* __restrict__ done) {
    constexpr int SUB = kJacobiThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double s_tool[3];
    if (int(blockIdx.x) >= n_list) return;
    const int env = env_list ? env_list[blockIdx.x] : int(blockIdx.x);
    const int st = threadIdx.x;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const int V = M.V, Vp = M.Vp, E = M.E, T = M.T;
    const long long stride = S.stride;
    const JacobiLayout L(Vp);
    float4* X = reinterpret_cast<float4*>(smem_raw + L.x);
    float* Ax = reinterpret_cast<float*>(smem_raw + L.acc);
    float* Ay = Ax + Vp;
    float* Az = Ay + Vp;
    unsigned* bits = reinterpret_cast<unsigned*>(smem_raw + L.bits);
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;
    for (int w = st; w < Vp / 32; w += SUB) bits[w] = 0u;
    for (int s = st; s < Vp; s += SUB) {
        Ax[s] = 0.f;
        Ay[s] = 0.f;
        Az[s] = 0.f;
    }
    if (st == 0) {
        // Tool update once per step (Algorithm 1), rounded product then sum.
        const unsigned long long t = (unsigned long long)S.t_step[env];
        const unsigned long long rs = env_stream(S.seed[env], ed.gid, 0u);
        for (int k = 0; k < 3; ++k) {
            const double a = actions ? (double)actions[3 * env + k] : to_unit_pm1(splitmix64_nth(rs, 3ull * t + k));
            double c = __dadd_rn(S.tool[3 * env + k], __dmul_rn(S.action_scale, a));
            c = c < M.box_lo[k] ? M.box_lo[k] : c;
            c = c > M.box_hi[k] ? M.box_hi[k] : c;
            S.tool[3 * env + k] = c;
            s_tool[k] = c;
        }
    }
    const float h = S.h, inv_h = S.inv_h;
    const float hgx = __fmul_rn(h, S.gx), hgy = __fmul_rn(h, S.gy), hgz = __fmul_rn(h, S.gz);
    {
        const float* gx = S.x + ed.voff;
        const float* gv = S.v + ed.voff;
        for (int i = st; i < V; i += SUB) {
            const int s = M.slot_of[i];
            float4 xi = make_float4(gx[i], gx[stride + i], gx[2 * stride + i], M.rest_w[i].w);
            Px[s] = xi.x;
            Py[s] = xi.y;
            Pz[s] = xi.z;
            if (xi.w > 0.f) {   // rounding spelled out, as in the single-CTA kernel
                xi.x = __fmaf_rn(h, __fadd_rn(gv[i], hgx), xi.x);
                xi.y = __fmaf_rn(h, __fadd_rn(gv[stride + i], hgy), xi.y);
                xi.z = __fmaf_rn(h, __fadd_rn(gv[2 * stride + i], hgz), xi.z);
            }
            X[s] = xi;
        }
    }
    __syncthreads();
    const float cx = float(s_tool[0]), cy = float(s_tool[1]), cz = float(s_tool[2]);
    const float rad = S.radius, rad2 = __fmul_rn(rad, rad);
    const float at_d = ed.alpha_d, at_v = S.alpha_v;
    float* lam = S.lambda ? S.lambda + ed.loff : nullptr;   // edges at [0, E), tets at [E, E + T)

    for (int sub = 0; sub < S.substeps; ++sub) {
        for (int it = 0; it < S.iterations; ++it) {
            const bool carry = lam != nullptr;
#pragma unroll 2
            for (int q = st; q < E; q += SUB) {
                const uint2 rec = __ldg(M.erec + q);
                float l = (carry && it > 0) ? lam[q] : 0.f;
                float3 da, db;
                edge_delta(X, rec, at_d, M.min_len2, l, da, db);
                if (carry) lam[q] = l;
                const int a = int(rec.x & 0xffffu), b = int(rec.x >> 16);
                atomicAdd(&Ax[a], da.x);
                atomicAdd(&Ay[a], da.y);
                atomicAdd(&Az[a], da.z);
                atomicAdd(&Ax[b], db.x);
                atomicAdd(&Ay[b], db.y);
                atomicAdd(&Az[b], db.z);
            }
#pragma unroll 2
            for (int q = st; q < T; q += SUB) {
                const uint4 rec = __ldg(M.trec + q);
                float l = (carry && it > 0) ? lam[E + q] : 0.f;
                float3 dx[4];
                tet_delta(X, rec, at_v, l, dx);
                if (carry) lam[E + q] = l;
                const int v4[4] = {int(rec.x & 0xffffu), int(rec.x >> 16), int(rec.y & 0xffffu), int(rec.y >> 16)};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    atomicAdd(&Ax[v4[i]], dx[i].x);
                    atomicAdd(&Ay[v4[i]], dx[i].y);
                    atomicAdd(&Az[v4[i]], dx[i].z);
                }
            }
            __syncthreads();
            // x_i += (sum of corrections) / n_i; the sums start again from zero
            for (int s = st; s < V; s += SUB) {
                const float f = M.inv_ncons[s];
                float4 xi = X[s];
                xi.x += Ax[s] * f;
                xi.y += Ay[s] * f;
                xi.z += Az[s] * f;
                X[s] = xi;
                Ax[s] = 0.f;
                Ay[s] = 0.f;
                Az[s] = 0.f;
            }
            __syncthreads();
        }
        // Collision, and except after the last substep the velocity update and
        // the next prediction (as the Gauss-Seidel kernel).
        const bool last = sub == S.substeps - 1;
        for (int s = st; s < V; s += SUB) {
            float4 xi = X[s];
            if (!(xi.w > 0.f)) {
                if (!last) {
                    Px[s] = xi.x;
                    Py[s] = xi.y;
                    Pz[s] = xi.z;
                }
                continue;
            }
            const float dx = __fsub_rn(xi.x, cx), dy = __fsub_rn(xi.y, cy), dz = __fsub_rn(xi.z, cz);
            const float l2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            if (l2 < rad2) {
                const float len = sqrtf(l2);
                if (len > 0.f) {
                    const float f = __fdividef(rad, len);
                    xi.x = __fmaf_rn(f, dx, cx);
                    xi.y = __fmaf_rn(f, dy, cy);
                    xi.z = __fmaf_rn(f, dz, cz);
                } else {
                    xi.x = cx;
                    xi.y = cy;
                    xi.z = __fadd_rn(cz, rad);
                }
                if (last) {
                    const int i = M.vert_of[s];
                    atomicOr(&bits[i >> 5], 1u << (i & 31));
                }
            }
            if (!last) {
                const float vx = __fmul_rn(__fsub_rn(xi.x, Px[s]), inv_h),
                            vy = __fmul_rn(__fsub_rn(xi.y, Py[s]), inv_h),
                            vz = __fmul_rn(__fsub_rn(xi.z, Pz[s]), inv_h);
                Px[s] = xi.x;
                Py[s] = xi.y;
                Pz[s] = xi.z;
                xi.x = __fmaf_rn(h, __fadd_rn(vx, hgx), xi.x);
                xi.y = __fmaf_rn(h, __fadd_rn(vy, hgy), xi.y);
                xi.z = __fmaf_rn(h, __fadd_rn(vz, hgz), xi.z);
            }
            X[s] = xi;
        }
        __syncthreads();
    }
    // Write back x and v = (x - x_prev) / h in vertex order; flag non-finite positions.
    float* ox = S.x + ed.voff;
    float* ov = S.v + ed.voff;
    bool bad = false;
    for (int i = st; i < V; i += SUB) {
        const int s = M.slot_of[i];
        const float4 xi = X[s];
        ox[i] = xi.x;
        ox[stride + i] = xi.y;
        ox[2 * stride + i] = xi.z;
        ov[i] = __fmul_rn(__fsub_rn(xi.x, Px[s]), inv_h);
        ov[stride + i] = __fmul_rn(__fsub_rn(xi.y, Py[s]), inv_h);
        ov[2 * stride + i] = __fmul_rn(__fsub_rn(xi.z, Pz[s]), inv_h);
        bad |= !(isfinite(xi.x) && isfinite(xi.y) && isfinite(xi.z));
    }
    if (bad) atomicOr(&S.err[env], kErrNonFinite);
    // Contacts of the last substep (ascending vertex ids), observation, reward, termination.
    const int lane = st & 31, warp = st >> 5;
    if (warp == 0) {
        const int nwords = Vp / 32;
        int base = 0;
        for (int w0 = 0; w0 < nwords; w0 += 32) {
            unsigned word = (w0 + lane < nwords) ? bits[w0 + lane] : 0u;
            const int cnt = __popc(word);
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int pos = base + incl - cnt;
            while (word) {
                const int bit = __ffs(word) - 1;
                word &= word - 1;
                S.contacts[ed.voff + pos++] = (w0 + lane) * 32 + bit;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) S.n_contacts[env] = base;
    }
    if (obs) {
        float* o = obs + (long long)env * S.obs_dim;
        const int* ids = S.obs_ids + (long long)env * S.n_obs;
        for (int j = st; j < S.obs_dim; j += SUB) {
            float val;
            if (j < 3) {
                val = float(s_tool[j]);
            } else {
                const int q = (j - 3) / 3, kk = (j - 3) - 3 * q;
                const float4 xv = X[M.slot_of[ids[q]]];
                val = kk == 0 ? xv.x : (kk == 1 ? xv.y : xv.z);
            }
            o[j] = val;
        }
    }
    if (st == 0) {
        const float4 xt = X[M.slot_of[S.target[env]]];
        const double dx = s_tool[0] - double(xt.x), dy = s_tool[1] - double(xt.y), dz = s_tool[2] - double(xt.z);
        const double l = sqrt(dx * dx + dy * dy + dz * dz);
        const int succ = l < S.success_dist;
        const double R = S.w_l * l + S.w_d * (l - double(S.l_prev[env])) + S.w_s * double(succ);
        S.l_prev[env] = float(l);
        const int t = S.t_step[env] + 1;
        S.t_step[env] = t;
        const uint8_t dn = uint8_t(((S.max_steps > 0 && t >= S.max_steps) || succ) ? 1 : 0);
        S.done_flag[env] = dn;
        if (reward) reward[env] = float(R);
        if (done) done[env] = dn;
    }
}

cudaError_t configure_jacobi_step(size_t smem) {
    static size_t configured = 48 * 1024;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(xpbd_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    return cudaSuccess;
}

cudaError_t launch_jacobi_step(const SimDev& S, const int* env_list, int n_list, size_t smem, cudaStream_t st,
                               const float* a, float* o, float* r, uint8_t* d) {
    if (n_list <= 0) return cudaSuccess;
    const cudaError_t ce = configure_jacobi_step(smem);
    if (ce != cudaSuccess) return ce;
    xpbd_jacobi_kernel<<<n_list, kJacobiThreads, smem, st>>>(S, env_list, n_list, a, o, r, d);
    return cudaGetLastError();
}

}  // namespace ffsrl
