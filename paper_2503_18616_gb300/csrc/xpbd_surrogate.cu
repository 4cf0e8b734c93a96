// Surrogate-assisted XPBD substeps (the learned warm-start of the workload;
// not in the FF-SRL paper, which runs the plain substep of Algorithm 1).
//
// One substep of every env is three launches: the features kernel (per
// vertex: displacement from rest, velocity, 1-ring mean position and
// velocity as offsets, offset from the tool, all at the predicted state),
// the tensor-core network (mlp_tc.cu), and the substep kernel below. The
// substep kernel predicts, adds the network's correction to free vertices,
// runs one constraint iteration, takes the largest relative constraint
// violation of the env, and if it exceeds the threshold restores the
// prediction and runs the full solve instead; then the tool collision and the
// velocity update (Algorithm 1), and on the last substep the observation,
// reward and termination. A record mode runs the full solve and writes the
// training targets (positions after the solve minus the prediction).
//
// The state goes through HBM between substeps (the features of the next
// substep need every vertex of the env), unlike the resident plain step.
#include <cstdint>

#include "xpbd_device.cuh"
#include "xpbd_project.cuh"
#include "xpbd_surrogate.h"

namespace ffsrl {

namespace {

// Tool update once per step (Algorithm 1, "evaluate instrument state"), as in
// the plain step kernel: rounded float64 product and sum, clamped to the box.
__device__ void update_tool(const SimDev& S, const MeshDev& M, int env, const float* actions, double* c_out) {
    const unsigned long long t = (unsigned long long)S.t_step[env];
    const unsigned long long rs = env_stream(S.seed[env], (unsigned long long)env, 0u);
    for (int k = 0; k < 3; ++k) {
        const double a = actions ? (double)actions[3 * env + k] : to_unit_pm1(splitmix64_nth(rs, 3ull * t + k));
        double c = __dadd_rn(S.tool[3 * env + k], __dmul_rn(S.action_scale, a));
        c = c < M.box_lo[k] ? M.box_lo[k] : c;
        c = c > M.box_hi[k] ? M.box_hi[k] : c;
        S.tool[3 * env + k] = c;
        c_out[k] = c;
    }
}

// Predicted position and velocity of vertex i (Algorithm 1): free vertices
// get v + h g and x + h (v + h g); pinned ones keep x and v.
__device__ __forceinline__ void predict_vertex(const SimDev& S, const MeshDev& M, int voff, int i, float3& xh,
                                               float3& vh) {
    const long long st = S.stride;
    const float* gx = S.x + voff;
    const float* gv = S.v + voff;
    xh = make_float3(gx[i], gx[st + i], gx[2 * st + i]);
    vh = make_float3(gv[i], gv[st + i], gv[2 * st + i]);
    if (M.rest_w[i].w > 0.f) {
        vh.x += S.h * S.gx;
        vh.y += S.h * S.gy;
        vh.z += S.h * S.gz;
        xh.x += S.h * vh.x;
        xh.y += S.h * vh.y;
        xh.z += S.h * vh.z;
    }
}

}  // namespace

// Features of every vertex at the predicted state of the coming substep;
// row voff + i of F holds 16 floats (15 features and a zero).
__global__ void __launch_bounds__(256) features_kernel(SimDev S, const int* __restrict__ env_list, int n_list,
                                                       int update, const float* __restrict__ actions,
                                                       float4* __restrict__ F) {
    __shared__ double s_c[3];
    if (int(blockIdx.x) >= n_list) return;
    const int env = env_list ? env_list[blockIdx.x] : int(blockIdx.x);
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    if (threadIdx.x == 0) {
        if (update) {
            update_tool(S, M, env, actions, s_c);
        } else {
            for (int k = 0; k < 3; ++k) s_c[k] = S.tool[3 * env + k];
        }
    }
    __syncthreads();
    const float cx = float(s_c[0]), cy = float(s_c[1]), cz = float(s_c[2]);
    for (int i = threadIdx.x; i < M.V; i += blockDim.x) {
        float3 xh, vh;
        predict_vertex(S, M, ed.voff, i, xh, vh);
        float3 mx = make_float3(0.f, 0.f, 0.f), mv = make_float3(0.f, 0.f, 0.f);
        const int b = M.nbr_off[i], e = M.nbr_off[i + 1];
        for (int q = b; q < e; ++q) {
            float3 xj, vj;
            predict_vertex(S, M, ed.voff, M.nbr[q], xj, vj);
            mx.x += xj.x; mx.y += xj.y; mx.z += xj.z;
            mv.x += vj.x; mv.y += vj.y; mv.z += vj.z;
        }
        const float inv = e > b ? 1.0f / float(e - b) : 0.f;
        const float4 r = M.rest_w[i];
        float4* f = F + 4 * (long long)(ed.voff + i);
        const float ox = e > b ? mx.x * inv - xh.x : 0.f, oy = e > b ? mx.y * inv - xh.y : 0.f,
                    oz = e > b ? mx.z * inv - xh.z : 0.f;
        const float wx = e > b ? mv.x * inv - vh.x : 0.f, wy = e > b ? mv.y * inv - vh.y : 0.f,
                    wz = e > b ? mv.z * inv - vh.z : 0.f;
        f[0] = make_float4(xh.x - r.x, xh.y - r.y, xh.z - r.z, vh.x);
        f[1] = make_float4(vh.y, vh.z, ox, oy);
        f[2] = make_float4(oz, wx, wy, wz);
        f[3] = make_float4(xh.x - cx, xh.y - cy, xh.z - cz, 0.f);
    }
}

namespace {

// `n_iter` constraint iterations of one env, records read from L2; lam (may
// be null for n_iter == 1) carries the multipliers across iterations.
template <int SUB>
__device__ void iterate(float4* X, const MeshDev& M, int n_iter, float at_d, float at_v, float* lam) {
    const int st = threadIdx.x;
    for (int it = 0; it < n_iter; ++it) {
        for (int c = 0; c < M.n_seg; ++c) {
            const int4 sg = M.segs[c];
            const unsigned char* base = M.recs + sg.x;
            if (c < M.n_ecol) {
                const uint2* rec = reinterpret_cast<const uint2*>(base);
                for (int q = st; q < sg.z; q += SUB) {
                    float l = (lam && it > 0) ? lam[sg.w + q] : 0.f;
                    project_edge(X, __ldg(rec + q), at_d, M.min_len2, l);
                    if (lam) lam[sg.w + q] = l;
                }
            } else {
                const uint4* rec = reinterpret_cast<const uint4*>(base);
                for (int q = st; q < sg.z; q += SUB) {
                    float l = (lam && it > 0) ? lam[sg.w + q] : 0.f;
                    project_tet(X, __ldg(rec + q), at_v, l);
                    if (lam) lam[sg.w + q] = l;
                }
            }
            __syncthreads();
        }
    }
}

// Largest relative violation (|C| / d, |C| / |V0|) over the env's
// constraints, reduced over the CTA (the result is the same in every thread).
template <int SUB>
__device__ float env_residual(const float4* X, const MeshDev& M, int* s_max) {
    const int st = threadIdx.x;
    float r = 0.f;
    for (int c = 0; c < M.n_seg; ++c) {
        const int4 sg = M.segs[c];
        const unsigned char* base = M.recs + sg.x;
        if (c < M.n_ecol) {
            for (int q = st; q < sg.z; q += SUB)
                r = fmaxf(r, edge_violation(X, __ldg(reinterpret_cast<const uint2*>(base) + q)));
        } else {
            for (int q = st; q < sg.z; q += SUB)
                r = fmaxf(r, tet_violation(X, __ldg(reinterpret_cast<const uint4*>(base) + q)));
        }
    }
    // non-negative floats order like their bit patterns; NaN maps above +inf
    atomicMax(s_max, isnan(r) ? 0x7f800001 : __float_as_int(r));
    __syncthreads();
    const float out = __int_as_float(*s_max);
    __syncthreads();
    return out;
}

}  // namespace

template <int SUB, bool RES>
__global__ void __launch_bounds__(SUB) substep_kernel(SimDev S, SubstepCtl C, const int* __restrict__ env_list,
                                                      int n_list, float* __restrict__ obs, float* __restrict__ reward,
                                                      uint8_t* __restrict__ done) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_red;
    __shared__ int s_resid;
    const int env = env_list[blockIdx.x];
    const int st = threadIdx.x;
    const EnvDev ed = S.envs[env];
    const MeshDev M = S.meshes[ed.mesh];
    const int V = M.V, Vp = M.Vp;
    const long long stride = S.stride;
    float4* X = RES ? reinterpret_cast<float4*>(smem_raw) : S.xg + ed.voff;
    unsigned* bits = reinterpret_cast<unsigned*>(smem_raw + (RES ? size_t(Vp) * 16 : 0));
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;
    const float inv_h = S.inv_h;
    const double cxd = S.tool[3 * env], cyd = S.tool[3 * env + 1], czd = S.tool[3 * env + 2];
    const float cx = float(cxd), cy = float(cyd), cz = float(czd);
    for (int w = st; w < Vp / 32; w += SUB) bits[w] = 0u;
    if (st == 0) {
        s_red = 0;
        s_resid = 0;
    }

    // Load and predict (vertex order in, slot order in X); add the correction.
    for (int i = st; i < V; i += SUB) {
        const int s = M.slot_of[i];
        float3 xh, vh;
        predict_vertex(S, M, ed.voff, i, xh, vh);
        const float w = M.rest_w[i].w;
        Px[s] = S.x[ed.voff + i];
        Py[s] = S.x[stride + ed.voff + i];
        Pz[s] = S.x[2 * stride + ed.voff + i];
        float4 xi = make_float4(xh.x, xh.y, xh.z, w);
        if (C.mode == kSubstepSurrogate && w > 0.f) {
            const float4 d = C.dx[ed.voff + i];
            xi.x += d.x;
            xi.y += d.y;
            xi.z += d.z;
        }
        X[s] = xi;
    }
    __syncthreads();
    float* lam = C.lambda ? C.lambda + ed.loff : nullptr;
    if (C.mode == kSubstepSurrogate) {
        iterate<SUB>(X, M, 1, ed.alpha_d, S.alpha_v, nullptr);
        const float r = env_residual<SUB>(X, M, &s_resid);
        if (st == 0 && C.residual) C.residual[env] = fmaxf(C.residual[env], r);
        if (!(r <= C.threshold)) atomicMax(&s_red, 1);   // a NaN residual also falls back
        __syncthreads();
        if (s_red) {
            // Fallback: back to the bare prediction, then the full solve.
            for (int i = st; i < V; i += SUB) {
                float3 xh, vh;
                predict_vertex(S, M, ed.voff, i, xh, vh);
                const int s = M.slot_of[i];
                X[s] = make_float4(xh.x, xh.y, xh.z, M.rest_w[i].w);
            }
            __syncthreads();
            iterate<SUB>(X, M, C.n_full, ed.alpha_d, S.alpha_v, lam);
            if (st == 0 && C.fallbacks) C.fallbacks[env] += 1;
        }
    } else {
        iterate<SUB>(X, M, C.n_full, ed.alpha_d, S.alpha_v, C.n_full > 1 ? lam : nullptr);
        if (C.residual) {
            const float r = env_residual<SUB>(X, M, &s_resid);
            if (st == 0) C.residual[env] = fmaxf(C.residual[env], r);
        }
        if (C.target) {
            for (int i = st; i < V; i += SUB) {
                float3 xh, vh;
                predict_vertex(S, M, ed.voff, i, xh, vh);
                const float4 xi = X[M.slot_of[i]];
                C.target[ed.voff + i] = make_float4(xi.x - xh.x, xi.y - xh.y, xi.z - xh.z, 0.f);
            }
        }
    }
    // Sphere-tool collision (Sec. III-A "Collisions").
    const float r = S.radius, r2 = r * r;
    for (int s = st; s < V; s += SUB) {
        float4 xi = X[s];
        if (!(xi.w > 0.f)) continue;
        const float dx = xi.x - cx, dy = xi.y - cy, dz = xi.z - cz;
        const float l2 = dx * dx + dy * dy + dz * dz;
        if (l2 < r2) {
            const float len = sqrtf(l2);
            if (len > 0.f) {
                const float f = __fdividef(r, len);
                xi.x = cx + f * dx;
                xi.y = cy + f * dy;
                xi.z = cz + f * dz;
            } else {
                xi.x = cx;
                xi.y = cy;
                xi.z = cz + r;
            }
            X[s] = xi;
            if (C.last) {
                const int i = M.vert_of[s];
                atomicOr(&bits[i >> 5], 1u << (i & 31));
            }
        }
    }
    __syncthreads();
    // Write back x and v = (x - x_prev) / h (vertex order).
    float* ox = S.x + ed.voff;
    float* ov = S.v + ed.voff;
    bool bad = false;
    for (int i = st; i < V; i += SUB) {
        const int s = M.slot_of[i];
        const float4 xi = X[s];
        ox[i] = xi.x;
        ox[stride + i] = xi.y;
        ox[2 * stride + i] = xi.z;
        ov[i] = (xi.x - Px[s]) * inv_h;
        ov[stride + i] = (xi.y - Py[s]) * inv_h;
        ov[2 * stride + i] = (xi.z - Pz[s]) * inv_h;
        bad |= !(isfinite(xi.x) && isfinite(xi.y) && isfinite(xi.z));
    }
    if (bad) atomicOr(&S.err[env], kErrNonFinite);
    if (!C.last) return;
    // Contacts of the last substep, observation, reward and termination.
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
                val = float(j == 0 ? cxd : (j == 1 ? cyd : czd));
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
        const double dx = cxd - double(xt.x), dy = cyd - double(xt.y), dz = czd - double(xt.z);
        const double l = sqrt(dx * dx + dy * dy + dz * dz);
        const int succ = l < S.success_dist;
        const double R = S.w_l * l + S.w_d * (l - double(S.l_prev[env])) + S.w_s * double(succ);
        S.l_prev[env] = float(l);
        const int t = S.t_step[env] + 1;
        S.t_step[env] = t;
        if (reward) reward[env] = float(R);
        if (done) done[env] = uint8_t(((S.max_steps > 0 && t >= S.max_steps) || succ) ? 1 : 0);
    }
}

size_t substep_smem_bytes(int Vp, bool resident) { return (resident ? size_t(Vp) * 16 : 0) + size_t(Vp / 32) * 4; }

cudaError_t launch_features(const SimDev& S, const int* env_list, int n_list, bool update_tool,
                            const float* actions, float4* F, cudaStream_t st) {
    if (n_list <= 0) return cudaSuccess;
    features_kernel<<<n_list, 256, 0, st>>>(S, env_list, n_list, update_tool ? 1 : 0, actions, F);
    return cudaGetLastError();
}

cudaError_t launch_substep(const SimDev& S, const SubstepCtl& C, const int* env_list, int n_list, bool resident,
                           size_t smem, cudaStream_t st, float* obs, float* reward, uint8_t* done) {
    if (n_list <= 0) return cudaSuccess;
    if (resident) {
        static size_t configured = 48 * 1024;
        if (smem > configured) {
            cudaError_t e = cudaFuncSetAttribute(substep_kernel<256, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            configured = smem;
        }
        substep_kernel<256, true><<<n_list, 256, smem, st>>>(S, C, env_list, n_list, obs, reward, done);
    } else {
        substep_kernel<256, false><<<n_list, 256, smem, st>>>(S, C, env_list, n_list, obs, reward, done);
    }
    return cudaGetLastError();
}

}  // namespace ffsrl
