// Surrogate-assisted XPBD substeps (a learned warm-start added to the method;
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

#include "tc_prims.cuh"
#include "xpbd_device.cuh"
#include "xpbd_project.cuh"
#include "xpbd_surrogate.h"

namespace ffsrl {

namespace {

// Maximum that keeps a NaN (fmaxf drops it): a NaN violation makes the
// residual NaN, which then falls back (the warm-start's residual reading).
__device__ __forceinline__ float nan_max(float r, float c) { return (isnan(c) || c > r) ? c : r; }

// Tool update once per step (Algorithm 1, "evaluate instrument state"), as in
// the plain step kernel: rounded float64 product and sum, clamped to the box.
__device__ void update_tool(const SimDev& S, const MeshDev& M, int env, const float* actions, double* c_out) {
    const unsigned long long t = (unsigned long long)S.t_step[env];
    const unsigned long long rs = env_stream(S.seed[env], S.envs[env].gid, 0u);
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
                r = nan_max(r, edge_violation(X, __ldg(reinterpret_cast<const uint2*>(base) + q)));
        } else {
            for (int q = st; q < sg.z; q += SUB)
                r = nan_max(r, tet_violation(X, __ldg(reinterpret_cast<const uint4*>(base) + q)));
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
        if (C.check) {
            const float r = env_residual<SUB>(X, M, &s_resid);
            if (st == 0 && C.residual) C.residual[env] = fmaxf(C.residual[env], r);
            if (C.decide && !(r <= C.threshold)) atomicMax(&s_red, 1);   // a NaN residual also falls back
        }
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
        const uint8_t dn = uint8_t(((S.max_steps > 0 && t >= S.max_steps) || succ) ? 1 : 0);
        S.done_flag[env] = dn;
        if (reward) reward[env] = float(R);
        if (done) done[env] = dn;
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

// ---- fused warm-start step ---------------------------------------------------
//
// One CTA of 256 threads advances one env through all substeps of a step with
// its positions resident in shared memory, as the plain step kernel does, and
// runs the warm-start network inside the same CTA on the tensor cores. Per
// substep: the features of every row (shared-memory slot) at the predicted
// state, the network tile by tile (128 rows: three tcgen05.mma chains into
// TMEM with the bias / ReLU / BF16 epilogues in between), the corrections
// added to the free vertices (every tile's features see the uncorrected
// prediction, as the method defines), one constraint iteration with the
// records streamed through a TMA double buffer, the residual sweep (order-free,
// records from L2) and the fallback to the full solve above the threshold,
// then collision, the velocity update and the next prediction.
//
// Two kernels implement it:
//   - warm_step_jit_kernel (meshes whose 1-ring spans at most four 128-row
//     tiles of slots): warps 4-7 build each tile's input just in time, while
//     warps 0-3 run the previous tile's tensor-core chain and epilogues; a
//     tile's network output stays in TMEM (four 16-column slots) until no
//     later tile's features read its rows, and is then added to the
//     positions. No global scratch but the predicted velocities and the
//     substep-start positions.
//   - warm_step_kernel (any mesh that fits): the features of every row first,
//     written to global scratch in the operand layout, then the network tile
//     by tile with the corrections staged in global scratch.
// Shared memory holds the positions and one region used in turn by the record
// ring (constraint phases) and by the weight, hidden and input tiles (network
// phase), so three CTAs fit on an SM. Predicted velocities and substep-start
// positions live in global memory in slot order (L1/L2-resident while the CTA
// runs). The fallback rebuilds the prediction exactly: x~ = fma(h, v~, x_prev)
// is the same rounded operation that made it. The two kernels give the same
// bits.
namespace {

constexpr int kNetBytes = kMlpWeightBytes + 16384;   // weight tiles + one hidden tile
constexpr int kJitNetBytes = kNetBytes + 4096;        // + one input tile
constexpr int kJitSlots = 4;                          // TMEM slots of pending network outputs

struct WarmLayout {
    size_t x, u, bias, segs, bits, total;
    __host__ __device__ WarmLayout(int Vp, int ring_bytes, int n_seg) {
        x = 0;
        u = size_t(Vp) * 16;
        const size_t un = 2 * size_t(ring_bytes) > size_t(kNetBytes) ? 2 * size_t(ring_bytes) : size_t(kNetBytes);
        bias = u + (un + 127) / 128 * 128;
        segs = bias + 144 * 4;
        bits = segs + size_t(n_seg) * 16;
        total = bits + size_t(Vp / 32) * 4;
    }
};

// The just-in-time kernel reads the segment table from L2 instead of shared
// memory (the room goes to the input tile).
struct JitLayout {
    size_t x, u, bias, bits, total;
    __host__ __device__ JitLayout(int Vp, int ring_bytes) {
        x = 0;
        u = size_t(Vp) * 16;
        const size_t un =
            2 * size_t(ring_bytes) > size_t(kJitNetBytes) ? 2 * size_t(ring_bytes) : size_t(kJitNetBytes);
        bias = u + (un + 127) / 128 * 128;
        bits = bias + 144 * 4;
        total = bits + size_t(Vp / 32) * 4;
    }
};

constexpr uint32_t kWarmTmemCols = 128;

// n_proj ring-buffered projection passes over the constraint records, colour
// by colour (multipliers carried in lam when n_proj > 1). Copy k of the step's
// running count goes to stage k & 1; one copy is in flight ahead of the colour
// being processed. Returns false (uniformly) if a copy did not arrive within
// the bounded wait.
__device__ bool ring_sweep(float4* X, const MeshDev& M, const int4* segs, unsigned char* ring, uint64_t* mbar,
                           uint32_t& k, int n_proj, float at_d, float at_v, float* lam) {
    using namespace tc;
    const int st = threadIdx.x;
    const int n_seg = M.n_seg, n_ecol = M.n_ecol;
    const int K = n_proj * n_seg;
    if (K == 0) return true;
    fence_async_smem();   // generic writes to the region before the copies overwrite it
    __syncthreads();
    if (st == 0) {
        const int4 sg = segs[0];
        mbar_expect_tx(&mbar[k & 1], uint32_t(sg.y));
        bulk_copy_g2s(ring + (k & 1) * M.ring_bytes, M.recs + sg.x, uint32_t(sg.y), &mbar[k & 1]);
    }
    for (int j = 0; j < K; ++j, ++k) {
        const int pass = j / n_seg, c = j - pass * n_seg;
        if (st == 0 && j + 1 < K) {
            const int cn = c + 1 == n_seg ? 0 : c + 1;
            const int4 nx = segs[cn];
            uint64_t* b = &mbar[(k + 1) & 1];
            mbar_expect_tx(b, uint32_t(nx.y));
            bulk_copy_g2s(ring + ((k + 1) & 1) * M.ring_bytes, M.recs + nx.x, uint32_t(nx.y), b);
        }
        const bool ok = mbar_wait(&mbar[k & 1], (k >> 1) & 1);
        if (ok) {
            const int4 sg = segs[c];
            const unsigned char* base = ring + (k & 1) * M.ring_bytes;
            const bool carry = lam != nullptr && n_proj > 1;
            // one pass keeps no multipliers: loops without their loads and stores
            if (c < n_ecol) {
                const uint2* rec = reinterpret_cast<const uint2*>(base);
                if (!carry) {
                    for (int q = st; q < sg.z; q += kWarmThreads) {
                        float l = 0.f;
                        project_edge(X, rec[q], at_d, M.min_len2, l);
                    }
                } else {
                    for (int q = st; q < sg.z; q += kWarmThreads) {
                        float l = pass > 0 ? lam[sg.w + q] : 0.f;
                        project_edge(X, rec[q], at_d, M.min_len2, l);
                        lam[sg.w + q] = l;
                    }
                }
            } else {
                const uint4* rec = reinterpret_cast<const uint4*>(base);
                if (!carry) {
                    for (int q = st; q < sg.z; q += kWarmThreads) {
                        float l = 0.f;
                        project_tet(X, rec[q], at_v, l);
                    }
                } else {
                    for (int q = st; q < sg.z; q += kWarmThreads) {
                        float l = pass > 0 ? lam[sg.w + q] : 0.f;
                        project_tet(X, rec[q], at_v, l);
                        lam[sg.w + q] = l;
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            // drain the copy that may still be in flight (bounded) before leaving
            if (st == 0 && j + 1 < K) mbar_wait(&mbar[(k + 1) & 1], ((k + 1) >> 1) & 1);
            ++k;
            return false;
        }
    }
    return true;
}

// Loads the env's state (vertex order in, slot order out), keeps the
// substep-start positions and predicts the first substep (Algorithm 1).
__device__ void warm_load_predict(const SimDev& S, const MeshDev& M, const EnvDev& ed, float4* X, float* Px,
                                  float* Py, float* Pz, float4* VH) {
    const long long stride = S.stride;
    const float h = S.h;
    const float hgx = h * S.gx, hgy = h * S.gy, hgz = h * S.gz;
    const float* gx = S.x + ed.voff;
    const float* gv = S.v + ed.voff;
    for (int i = threadIdx.x; i < M.V; i += kWarmThreads) {
        const int s = M.slot_of[i];
        const float w = M.rest_w[i].w;
        const float x0 = gx[i], x1 = gx[stride + i], x2 = gx[2 * stride + i];
        float v0 = gv[i], v1 = gv[stride + i], v2 = gv[2 * stride + i];
        Px[s] = x0;
        Py[s] = x1;
        Pz[s] = x2;
        if (w > 0.f) {
            v0 += hgx;
            v1 += hgy;
            v2 += hgz;
            X[s] = make_float4(__fmaf_rn(h, v0, x0), __fmaf_rn(h, v1, x1), __fmaf_rn(h, v2, x2), w);
        } else {
            X[s] = make_float4(x0, x1, x2, w);
        }
        VH[s] = make_float4(v0, v1, v2, 0.f);
    }
}

// The per-row tables the features of slot s read from global memory (its
// 1-ring header and neighbour slots, its rest position), loaded ahead of use.
struct FeatRow {
    uint4 c0, c1, c2;   // the slot's 1-ring record: degree, then neighbour slots (uint16 fields)
    float4 rest;
};

__device__ __forceinline__ FeatRow warm_feat_fetch(const MeshDev& M, int s) {
    FeatRow r;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    r.c0 = r.c1 = r.c2 = zero;
    r.rest = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < M.V) {
        const uint4* rec = M.snbr + 3 * s;
        r.c0 = __ldg(rec);
        r.c1 = __ldg(rec + 1);
        r.c2 = __ldg(rec + 2);
        r.rest = __ldg(M.rest_s + s);
    }
    return r;
}

// Features of slot s (15 values, normalised, the 16th zero) packed as BF16
// pairs from its tables; rows s >= V give zeros.
__device__ __forceinline__ void warm_features_row(const MeshDev& M, const MlpDev& net, const float4* X,
                                                  const float4* VH, int s, const FeatRow& r, float cx, float cy,
                                                  float cz, uint32_t* pk) {
    using namespace tc;
    float f[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) f[q] = 0.f;
    if (s < M.V) {
        const float4 xs = X[s];
        const float4 vs = VH[s];
        const uint32_t w[12] = {r.c0.x, r.c0.y, r.c0.z, r.c0.w, r.c1.x, r.c1.y,
                                r.c1.z, r.c1.w, r.c2.x, r.c2.y, r.c2.z, r.c2.w};
        const int deg = int(w[0] & 0xFFFF);
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
        for (int q = 0; q < kWarmMaxDegree; ++q) {
            if (q < deg) {
                const int j = (w[(q + 1) >> 1] >> (16 * ((q + 1) & 1))) & 0xFFFF;
                const float4 xj = X[j];
                const float4 vj = VH[j];
                m0 += xj.x; m1 += xj.y; m2 += xj.z;
                n0 += vj.x; n1 += vj.y; n2 += vj.z;
            }
        }
        const float4 rs = r.rest;
        f[0] = xs.x - rs.x; f[1] = xs.y - rs.y; f[2] = xs.z - rs.z;
        f[3] = vs.x; f[4] = vs.y; f[5] = vs.z;
        if (deg > 0) {
            const float inv = 1.0f / float(deg);
            f[6] = m0 * inv - xs.x; f[7] = m1 * inv - xs.y; f[8] = m2 * inv - xs.z;
            f[9] = n0 * inv - vs.x; f[10] = n1 * inv - vs.y; f[11] = n2 * inv - vs.z;
        }
        f[12] = xs.x - cx; f[13] = xs.y - cy; f[14] = xs.z - cz;
#pragma unroll
        for (int q = 0; q < 15; ++q) f[q] = (f[q] - net.in_mean[q]) * net.in_inv_std[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) pk[q] = pack_bf16x2(f[2 * q], f[2 * q + 1]);
}

__device__ __forceinline__ void warm_features(const MeshDev& M, const MlpDev& net, const float4* X, const float4* VH,
                                              int s, float cx, float cy, float cz, uint32_t* pk) {
    warm_features_row(M, net, X, VH, s, warm_feat_fetch(M, s), cx, cy, cz, pk);
}

// Bias, ReLU and BF16 rounding of 16 accumulator columns c0 .. c0+15 of this
// thread's row into the hidden tile (K-major, 64 columns).
__device__ __forceinline__ void warm_hidden16(uint32_t taddr, const float* bias, int c0, unsigned char* Ht,
                                              int erow) {
    using namespace tc;
    float v[16];
    tmem_ld16(taddr, v);
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        pk[q] = pack_bf16x2_relu(v[2 * q] + bias[c0 + 2 * q], v[2 * q + 1] + bias[c0 + 2 * q + 1]);
    *reinterpret_cast<uint4*>(Ht + tile_off(erow, c0 / 8, 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(Ht + tile_off(erow, c0 / 8 + 1, 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// The same for 32 columns c0 .. c0+31 (one TMEM load).
__device__ __forceinline__ void warm_hidden32(uint32_t taddr, const float* bias, int c0, unsigned char* Ht,
                                              int erow) {
    using namespace tc;
    float v[32];
    tmem_ld32(taddr, v);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = 16 * h + 2 * q;
            pk[q] = pack_bf16x2_relu(v[c] + bias[c0 + c], v[c + 1] + bias[c0 + c + 1]);
        }
        *reinterpret_cast<uint4*>(Ht + tile_off(erow, c0 / 8 + 2 * h, 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4*>(Ht + tile_off(erow, c0 / 8 + 2 * h + 1, 8)) =
            make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
}

// The de-normalised network output (3 accumulator columns from v) of slot s
// added to a free vertex.
__device__ __forceinline__ void warm_correct(float4* X, const MlpDev& net, const float* bias, int s, int V,
                                             const float* v) {
    if (s >= V) return;
    float4 xi = X[s];
    if (!(xi.w > 0.f)) return;
    const float y0 = (v[0] + bias[128]) * net.out_std[0] + net.out_mean[0];
    const float y1 = (v[1] + bias[129]) * net.out_std[1] + net.out_mean[1];
    const float y2 = (v[2] + bias[130]) * net.out_std[2] + net.out_mean[2];
    xi.x += y0;
    xi.y += y1;
    xi.z += y2;
    X[s] = xi;
}

// Sphere collision (Sec. III-A "Collisions"), the velocity update and the
// next substep's prediction (Algorithm 1), two vertices per thread and trip
// with their global loads issued together; on the last substep only the
// collision, with the contact bits.
__device__ void warm_collide_advance(const SimDev& S, const MeshDev& M, float4* X, float* Px, float* Py, float* Pz,
                                     float4* VH, unsigned* bits, float cx, float cy, float cz, bool last) {
    constexpr int SUB = kWarmThreads;
    const int V = M.V;
    const float h = S.h, inv_h = S.inv_h;
    const float hgx = h * S.gx, hgy = h * S.gy, hgz = h * S.gz;
    const float rad = S.radius, rad2 = rad * rad;
    for (int s0 = threadIdx.x; s0 < V; s0 += 2 * SUB) {
        float4 xv[2];
        float p0[2], p1[2], p2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = s0 + u * SUB;
            if (s < V) {
                xv[u] = X[s];
                p0[u] = Px[s];
                p1[u] = Py[s];
                p2[u] = Pz[s];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = s0 + u * SUB;
            if (s >= V) continue;
            float4 xi = xv[u];
            const float w = xi.w;
            if (w > 0.f) {
                const float dx = xi.x - cx, dy = xi.y - cy, dz = xi.z - cz;
                const float l2 = dx * dx + dy * dy + dz * dz;
                if (l2 < rad2) {
                    const float len = sqrtf(l2);
                    if (len > 0.f) {
                        const float f = __fdividef(rad, len);
                        xi.x = cx + f * dx;
                        xi.y = cy + f * dy;
                        xi.z = cz + f * dz;
                    } else {
                        xi.x = cx;
                        xi.y = cy;
                        xi.z = cz + rad;
                    }
                    if (last) {
                        const int i = M.vert_of[s];
                        atomicOr(&bits[i >> 5], 1u << (i & 31));
                    }
                }
            }
            if (last) {
                X[s] = xi;
                continue;
            }
            float v0 = (xi.x - p0[u]) * inv_h, v1 = (xi.y - p1[u]) * inv_h, v2 = (xi.z - p2[u]) * inv_h;
            Px[s] = xi.x;
            Py[s] = xi.y;
            Pz[s] = xi.z;
            if (w > 0.f) {
                v0 += hgx;
                v1 += hgy;
                v2 += hgz;
                xi.x = __fmaf_rn(h, v0, xi.x);
                xi.y = __fmaf_rn(h, v1, xi.y);
                xi.z = __fmaf_rn(h, v2, xi.z);
            }
            VH[s] = make_float4(v0, v1, v2, 0.f);
            X[s] = xi;
        }
    }
}

// One constraint iteration, the residual sweep (when C.check) and the
// fallback to the full solve (when C.decide and the residual is not at most
// the threshold, NaN included). Returns false (uniformly) if a bounded wait
// gave up.
__device__ bool warm_iterate(const SimDev& S, const MeshDev& M, const EnvDev& ed, int env, const SubstepCtl& C,
                             float4* X, const float* Px, const float* Py, const float* Pz, const float4* VH,
                             const int4* segs, unsigned char* U, uint64_t* mbar, uint32_t& k, int* s_resid,
                             int& n_fallback) {
    constexpr int SUB = kWarmThreads;
    const int tid = threadIdx.x;
    const float h = S.h;
    if (!ring_sweep(X, M, segs, U, mbar, k, 1, ed.alpha_d, S.alpha_v, nullptr)) return false;
    float res = 0.f;
    if (C.check) {
        // it only reads positions, so it needs neither the colour order nor
        // barriers; the unpadded record lists come from L2
        float rmax = 0.f;
        const uint2* er = M.erec;
        const uint4* tr = M.trec;
#pragma unroll 4
        for (int q = tid; q < M.E; q += SUB) rmax = nan_max(rmax, edge_violation(X, __ldg(er + q)));
#pragma unroll 4
        for (int q = tid; q < M.T; q += SUB) rmax = nan_max(rmax, tet_violation(X, __ldg(tr + q)));
        // non-negative floats order like their bit patterns; NaN maps above +inf
        atomicMax(s_resid, isnan(rmax) ? 0x7f800001 : __float_as_int(rmax));
        __syncthreads();
        res = __int_as_float(*s_resid);
        if (tid == 0 && C.residual) C.residual[env] = fmaxf(C.residual[env], res);
    }
    if (C.decide && !(res <= C.threshold)) {   // uniform over the CTA
        for (int s = tid; s < M.V; s += SUB) {
            const float w = X[s].w;
            const float4 vh = VH[s];
            const float p0 = Px[s], p1 = Py[s], p2 = Pz[s];
            X[s] = w > 0.f ? make_float4(__fmaf_rn(h, vh.x, p0), __fmaf_rn(h, vh.y, p1), __fmaf_rn(h, vh.z, p2), w)
                           : make_float4(p0, p1, p2, w);
        }
        if (!ring_sweep(X, M, segs, U, mbar, k, C.n_full, ed.alpha_d, S.alpha_v,
                        C.lambda ? C.lambda + ed.loff : nullptr))
            return false;
        ++n_fallback;
    }
    return true;
}

// Writes x and v = (x - x_prev) / h back in vertex order (flagging non-finite
// positions), then the contacts of the last substep (ascending vertex ids),
// the observation, the reward and termination (Sec. III-B, Sec. IV).
__device__ void warm_write_outputs(const SimDev& S, const MeshDev& M, const EnvDev& ed, int env, const float4* X,
                                   const float* Px, const float* Py, const float* Pz, const unsigned* bits,
                                   const double* s_tool, float* obs, float* reward, uint8_t* done) {
    constexpr int SUB = kWarmThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long stride = S.stride;
    const float inv_h = S.inv_h;
    float* ox = S.x + ed.voff;
    float* ov = S.v + ed.voff;
    bool bad = false;
    for (int i = tid; i < M.V; i += SUB) {
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
    if (warp == 0) {
        const int nwords = M.Vp / 32;
        int base = 0;
        for (int w0 = 0; w0 < nwords; w0 += 32) {
            unsigned word = (w0 + lane < nwords) ? bits[w0 + lane] : 0u;
            const int cnt = __popc(word);
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int tt = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += tt;
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
        for (int j = tid; j < S.obs_dim; j += SUB) {
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
    if (tid == 0) {
        const float4 xt = X[M.slot_of[S.target[env]]];
        const double dx = s_tool[0] - double(xt.x), dy = s_tool[1] - double(xt.y), dz = s_tool[2] - double(xt.z);
        const double l = sqrt(dx * dx + dy * dy + dz * dz);
        const int succ = l < S.success_dist;
        const double R = S.w_l * l + S.w_d * (l - double(S.l_prev[env])) + S.w_s * double(succ);
        S.l_prev[env] = float(l);
        const int tt = S.t_step[env] + 1;
        S.t_step[env] = tt;
        const uint8_t dn = uint8_t(((S.max_steps > 0 && tt >= S.max_steps) || succ) ? 1 : 0);
        S.done_flag[env] = dn;
        if (reward) reward[env] = float(R);
        if (done) done[env] = dn;
    }
}

}  // namespace

size_t warm_smem_bytes(int Vp, int ring_bytes, int n_seg, bool jit) {
    return jit ? JitLayout(Vp, ring_bytes).total : WarmLayout(Vp, ring_bytes, n_seg).total;
}

__global__ void __launch_bounds__(kWarmThreads, 3)
    warm_step_kernel(SimDev S, MlpDev net, SubstepCtl C, const int* __restrict__ env_list, int n_list,
                     const float* __restrict__ actions, float* __restrict__ obs, float* __restrict__ reward,
                     uint8_t* __restrict__ done) {
    using namespace tc;
    constexpr int SUB = kWarmThreads;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[3];   // [0], [1] record ring; [2] tensor-core completion
    __shared__ uint32_t tmem_slot;
    __shared__ double s_tool[3];
    __shared__ int s_resid;
    if (int(blockIdx.x) >= n_list) return;
    const int env = env_list[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const int V = M.V, Vp = M.Vp;
    const long long stride = S.stride;
    const WarmLayout L(Vp, M.ring_bytes, M.n_seg);
    float4* X = reinterpret_cast<float4*>(sm + L.x);
    unsigned char* U = sm + L.u;            // record ring, or weight tiles + hidden tile
    unsigned char* Wt = U;
    unsigned char* Ht = U + kMlpWeightBytes;
    unsigned char* At = Ht;                 // the input tile is dead once layer 1 has read it
    float* bias = reinterpret_cast<float*>(sm + L.bias);
    int4* segs = reinterpret_cast<int4*>(sm + L.segs);
    unsigned* bits = reinterpret_cast<unsigned*>(sm + L.bits);
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;
    float4* DX = C.scratch + ed.voff;       // corrections, slot order
    float4* VH = C.vpred + ed.voff;         // predicted velocities, slot order
    uint4* AR = C.arows + 2 * (ed.voff + 128ll * env);   // network input tiles, 4 KB each

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kWarmTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 144; i += SUB) bias[i] = net.bias[i];
    for (int c = tid; c < M.n_seg; c += SUB) segs[c] = M.segs[c];
    for (int w = tid; w < Vp / 32; w += SUB) bits[w] = 0u;
    if (tid == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
        mbar_init(&mbar[2]);
        update_tool(S, M, env, actions, s_tool);
    }
    warm_load_predict(S, M, ed, X, Px, Py, Pz, VH);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc64 = umma_idesc_bf16(128, 64), idesc16 = umma_idesc_bf16(128, 16);
    const uint32_t aW1 = saddr(Wt), aW2 = aW1 + 2048, aW3 = aW1 + 10240, aA = saddr(At), aH = saddr(Ht);
    const float cx = float(s_tool[0]), cy = float(s_tool[1]), cz = float(s_tool[2]);
    const int n_tiles = (V + 127) / 128;
    // TMEM lanes of this warp (a warp reaches the 32 lanes of its quarter) and
    // the column half it reads back in the hidden-layer epilogues.
    const int q4 = warp & 3, chalf = warp >> 2;
    const uint32_t tlane = uint32_t(32 * q4) << 16;
    const int erow = 32 * q4 + lane;
    uint32_t phase = 0;   // tensor-core completions so far
    uint32_t k = 0;       // record copies so far
    bool failed = false;
    int n_fallback = 0;

    for (int sub = 0; sub < S.substeps && !failed; ++sub) {
        const bool last = sub == S.substeps - 1;
        if (tid == 0) s_resid = 0;
        // -- the weight tiles into the shared region (the ring used it last)
        for (int i = tid; i < kMlpWeightBytes / 16; i += SUB)
            reinterpret_cast<uint4*>(Wt)[i] = reinterpret_cast<const uint4*>(net.wtiles)[i];
        // -- features of every row at the predicted state, normalised and
        //    rounded to BF16, written as the network's input tiles (the
        //    tensor-core operand layout) to global scratch: one row per thread
        for (int s = tid; s < n_tiles * 128; s += SUB) {
            uint32_t pk[8];
            warm_features(M, net, X, VH, s, cx, cy, cz, pk);
            unsigned char* tile = reinterpret_cast<unsigned char*>(AR) + size_t(s >> 7) * 4096;
            *reinterpret_cast<uint4*>(tile + tile_off(s & 127, 0, 2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(tile + tile_off(s & 127, 1, 2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        __syncthreads();
        // -- the network, one 128-row tile at a time (the next tile's input
        //    is fetched into registers while the current tile runs)
        uint4 a_next = AR[tid];
        for (int t = 0; t < n_tiles; ++t) {
            reinterpret_cast<uint4*>(At)[tid] = a_next;
            if (t + 1 < n_tiles) a_next = AR[(t + 1) * 256 + tid];
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            // Layer 1: D[0:64) = A (128 x 16) W1^T.
            if (tid == 0) {
                umma_bf16(tmem, umma_desc(aA, 128, 256), umma_desc(aW1, 128, 256), idesc64, 0);
                umma_commit(&mbar[2]);
            }
            if (__syncthreads_or(!mbar_wait(&mbar[2], phase & 1))) {
                failed = true;
                break;
            }
            ++phase;
            fence_after_sync();
            // Epilogue 1: bias, ReLU, BF16 -> hidden tile (each warp: 32 rows x 32 columns).
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int c0 = 32 * chalf + 16 * c;
                warm_hidden16(tmem + tlane + c0, bias, c0, Ht, erow);
            }
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            // Layer 2: D[64:128) = H1 (128 x 64) W2^T, four K = 16 steps.
            if (tid == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    umma_bf16(tmem + 64, umma_desc(aH + 256 * j, 128, 1024), umma_desc(aW2 + 256 * j, 128, 1024),
                              idesc64, j);
                umma_commit(&mbar[2]);
            }
            if (__syncthreads_or(!mbar_wait(&mbar[2], phase & 1))) {
                failed = true;
                break;
            }
            ++phase;
            fence_after_sync();
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int c0 = 32 * chalf + 16 * c;
                warm_hidden16(tmem + tlane + 64 + c0, bias + 64, c0, Ht, erow);
            }
            fence_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            // Layer 3: D[0:16) = H2 (128 x 64) W3^T (rows 3..15 of W3 are zero).
            if (tid == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    umma_bf16(tmem, umma_desc(aH + 256 * j, 128, 1024), umma_desc(aW3 + 256 * j, 128, 1024), idesc16,
                              j);
                umma_commit(&mbar[2]);
            }
            if (__syncthreads_or(!mbar_wait(&mbar[2], phase & 1))) {
                failed = true;
                break;
            }
            ++phase;
            fence_after_sync();
            if (warp < 4) {
                float v[16];
                tmem_ld16(tmem + tlane, v);
                const int s = t * 128 + erow;
                if (s < V) {
                    const float y0 = (v[0] + bias[128]) * net.out_std[0] + net.out_mean[0];
                    const float y1 = (v[1] + bias[129]) * net.out_std[1] + net.out_mean[1];
                    const float y2 = (v[2] + bias[130]) * net.out_std[2] + net.out_mean[2];
                    DX[s] = make_float4(y0, y1, y2, 0.f);
                }
            }
            fence_before_sync();
            __syncthreads();   // the next tile overwrites the input tile and TMEM columns 0..63
            fence_after_sync();
        }
        if (failed) break;
        // -- corrections of the free vertices (the features above saw none of them)
        for (int s = tid; s < V; s += SUB) {
            float4 xi = X[s];
            if (xi.w > 0.f) {
                const float4 d = DX[s];
                xi.x += d.x;
                xi.y += d.y;
                xi.z += d.z;
                X[s] = xi;
            }
        }
        // -- one iteration, the residual and the fallback to the full solve
        if (!warm_iterate(S, M, ed, env, C, X, Px, Py, Pz, VH, segs, U, mbar, k, &s_resid, n_fallback)) {
            failed = true;
            break;
        }
        // -- collision, velocity update and the next prediction
        warm_collide_advance(S, M, X, Px, Py, Pz, VH, bits, cx, cy, cz, last);
        __syncthreads();
    }
    if (failed) {
        // A bounded wait gave up: let the tensor-core commit in flight land
        // (bounded), free TMEM, flag the env and leave its state.
        mbar_wait(&mbar[2], phase & 1);
        if (tid == 0) atomicOr(&S.err[env], kErrTimeout);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWarmTmemCols)
                     : "memory");
    if (failed) return;
    if (tid == 0 && C.fallbacks && n_fallback) C.fallbacks[env] += n_fallback;
    warm_write_outputs(S, M, ed, env, X, Px, Py, Pz, bits, s_tool, obs, reward, done);
}

// The just-in-time kernel. Warps 0-3 ("epilogue warps", one TMEM lane quarter
// each) run the tensor-core chain of tile t: layer 1 into TMEM columns 0..63,
// its epilogue into the hidden tile, layer 2 into columns 0..63 again, its
// epilogue, layer 3 into the pending slot 64 + 16 (t mod 4). Warps 4-7
// ("feature warps", one row each) meanwhile gather the features of tile t + 1
// and write them into the input tile once layer 1 of tile t has read it.
// The features of a tile read rows at most R = M.tile_reach tiles away, so the
// output of tile p is added to the positions at the start of tile p + r with
// r = max(R, 2) (every feature that reads its rows is built by then, and the
// commit waited on in tile p + r - 1 covers layer 3 of tile p); r <= 4 slots.
__global__ void __launch_bounds__(kWarmThreads, 3)
    warm_step_jit_kernel(SimDev S, MlpDev net, SubstepCtl C, const int* __restrict__ env_list, int n_list,
                         const float* __restrict__ actions, float* __restrict__ obs, float* __restrict__ reward,
                         uint8_t* __restrict__ done) {
    using namespace tc;
    constexpr int SUB = kWarmThreads;
    extern __shared__ __align__(1024) unsigned char sm[];
    // [0], [1] record ring; [2] tensor-core completions for the epilogue
    // warps; [3] layer-1 completions for the feature warps (input tile free)
    __shared__ __align__(8) uint64_t mbar[4];
    __shared__ uint32_t tmem_slot;
    __shared__ double s_tool[3];
    __shared__ int s_resid;
    if (int(blockIdx.x) >= n_list) return;
    const int env = env_list[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const int V = M.V, Vp = M.Vp;
    const long long stride = S.stride;
    const JitLayout L(Vp, M.ring_bytes);
    float4* X = reinterpret_cast<float4*>(sm + L.x);
    unsigned char* U = sm + L.u;            // record ring, or weight, hidden and input tiles
    unsigned char* Wt = U;
    unsigned char* Ht = U + kMlpWeightBytes;
    unsigned char* At = Ht + 16384;
    float* bias = reinterpret_cast<float*>(sm + L.bias);
    unsigned* bits = reinterpret_cast<unsigned*>(sm + L.bits);
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;
    float4* VH = C.vpred + ed.voff;         // predicted velocities, slot order

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(kWarmTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < 144; i += SUB) bias[i] = net.bias[i];
    for (int w = tid; w < Vp / 32; w += SUB) bits[w] = 0u;
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(&mbar[b]);
        update_tool(S, M, env, actions, s_tool);
    }
    warm_load_predict(S, M, ed, X, Px, Py, Pz, VH);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc64 = umma_idesc_bf16(128, 64), idesc16 = umma_idesc_bf16(128, 16);
    const uint32_t aW1 = saddr(Wt), aW2 = aW1 + 2048, aW3 = aW1 + 10240, aA = saddr(At), aH = saddr(Ht);
    const float cx = float(s_tool[0]), cy = float(s_tool[1]), cz = float(s_tool[2]);
    const int n_tiles = (V + 127) / 128;
    // tiles of pinned vertices only come first in slot order on meshes pinned
    // at their lowest vertex ids; their outputs would never be applied
    const int t0 = M.first_free_tile < n_tiles ? M.first_free_tile : n_tiles;
    const int reach = M.tile_reach > 2 ? M.tile_reach : 2;
    const bool epi = warp < 4;
    const uint32_t tlane = uint32_t(32 * (warp & 3)) << 16;
    const int erow = 32 * (warp & 3) + lane;   // epilogue warps: the tile row of this lane
    const int frow = tid - 128;                // feature warps: the tile row of this thread
    uint32_t ph_e = 0;    // completions of mbar[2] seen by the epilogue warps
    uint32_t ph_a = 0;    // completions of mbar[3] seen by the feature warps
    uint32_t k = 0;       // record copies so far
    bool failed = false;
    int n_fallback = 0;
    const int4* segs = M.segs;

    // network output of tile p (pending in its TMEM slot) added to the free vertices of its rows
    auto apply_tile = [&](int p) {
        float v[4];
        tmem_ld4(tmem + tlane + 64 + 16 * (p & (kJitSlots - 1)), v);
        warm_correct(X, net, bias, p * 128 + erow, V, v);
    };

    for (int sub = 0; sub < S.substeps && !failed; ++sub) {
        const bool last = sub == S.substeps - 1;
        if (tid == 0) s_resid = 0;
        // -- the weight tiles into the shared region (the ring used it last),
        //    and the input tile of tile 0
        for (int i = tid; i < kMlpWeightBytes / 16; i += SUB)
            reinterpret_cast<uint4*>(Wt)[i] = reinterpret_cast<const uint4*>(net.wtiles)[i];
        FeatRow fr{};   // feature warps: the tables of their row of the next tile, fetched a tile ahead
        if (!epi) {
            uint32_t pk[8];
            warm_features(M, net, X, VH, t0 * 128 + frow, cx, cy, cz, pk);
            *reinterpret_cast<uint4*>(At + tile_off(frow, 0, 2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(At + tile_off(frow, 1, 2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            fr = warm_feat_fetch(M, (t0 + 1) * 128 + frow);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        bool bad = false;
        for (int t = t0; t < n_tiles; ++t) {
            // Layer 1: D[0:64) = A (128 x 16) W1^T; its completion is signalled
            // to both warp groups.
            if (tid == 0) {
                umma_bf16(tmem, umma_desc(aA, 128, 256), umma_desc(aW1, 128, 256), idesc64, 0);
                umma_commit(&mbar[2]);
                umma_commit(&mbar[3]);
            }
            if (epi) {
                if (t - reach >= t0) apply_tile(t - reach);
                bad |= !mbar_wait(&mbar[2], ph_e & 1);
                ++ph_e;
                fence_after_sync();
#pragma unroll
                for (int c = 0; c < 2; ++c) warm_hidden32(tmem + tlane + 32 * c, bias, 32 * c, Ht, erow);
                fence_async_smem();
                fence_before_sync();
                named_bar_sync(1, 128);
                fence_after_sync();
                // Layer 2: D[0:64) = H1 (128 x 64) W2^T, four K = 16 steps (layer 1's
                // columns, read back above).
                if (tid == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        umma_bf16(tmem, umma_desc(aH + 256 * j, 128, 1024), umma_desc(aW2 + 256 * j, 128, 1024),
                                  idesc64, j);
                    umma_commit(&mbar[2]);
                }
                bad |= !mbar_wait(&mbar[2], ph_e & 1);
                ++ph_e;
                fence_after_sync();
#pragma unroll
                for (int c = 0; c < 2; ++c) warm_hidden32(tmem + tlane + 32 * c, bias + 64, 32 * c, Ht, erow);
                fence_async_smem();
                fence_before_sync();
                named_bar_sync(1, 128);
                fence_after_sync();
                // Layer 3: the pending slot of tile t = H2 (128 x 64) W3^T (rows
                // 3..15 of W3 are zero); read back r tiles later.
                if (tid == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        umma_bf16(tmem + 64 + 16 * (t & (kJitSlots - 1)), umma_desc(aH + 256 * j, 128, 1024),
                                  umma_desc(aW3 + 256 * j, 128, 1024), idesc16, j);
                }
            } else {
                uint32_t pk[8];
                if (t + 1 < n_tiles) {
                    warm_features_row(M, net, X, VH, (t + 1) * 128 + frow, fr, cx, cy, cz, pk);
                    fr = warm_feat_fetch(M, (t + 2) * 128 + frow);
                }
                // layer 1 of tile t has read the input tile once this completes
                bad |= !mbar_wait(&mbar[3], ph_a & 1);
                ++ph_a;
                if (t + 1 < n_tiles) {
                    *reinterpret_cast<uint4*>(At + tile_off(frow, 0, 2)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4*>(At + tile_off(frow, 1, 2)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    fence_async_smem();
                }
            }
            fence_before_sync();
            if (__syncthreads_or(bad)) {
                failed = true;
                break;
            }
            fence_after_sync();
        }
        if (failed) break;
        // -- the outputs of the last tiles, once layer 3 of the last tile is done
        if (tid == 0) umma_commit(&mbar[2]);
        if (epi) {
            bad |= !mbar_wait(&mbar[2], ph_e & 1);
            ++ph_e;
            fence_after_sync();
            for (int p = n_tiles - reach > t0 ? n_tiles - reach : t0; p < n_tiles; ++p) apply_tile(p);
        }
        fence_before_sync();
        if (__syncthreads_or(bad)) {
            failed = true;
            break;
        }
        fence_after_sync();
        // -- one iteration, the residual and the fallback to the full solve
        if (!warm_iterate(S, M, ed, env, C, X, Px, Py, Pz, VH, segs, U, mbar, k, &s_resid, n_fallback)) {
            failed = true;
            break;
        }
        // -- collision, velocity update and the next prediction
        warm_collide_advance(S, M, X, Px, Py, Pz, VH, bits, cx, cy, cz, last);
        __syncthreads();
    }
    if (failed) {
        // A bounded wait gave up: one more commit covers every tensor-core
        // operation issued so far; let it land (bounded), free TMEM, flag the
        // env and leave its state.
        if (tid == 0) umma_commit(&mbar[2]);
        if (epi) mbar_wait(&mbar[2], ph_e & 1);
        if (tid == 0) atomicOr(&S.err[env], kErrTimeout);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWarmTmemCols)
                     : "memory");
    if (failed) return;
    if (tid == 0 && C.fallbacks && n_fallback) C.fallbacks[env] += n_fallback;
    warm_write_outputs(S, M, ed, env, X, Px, Py, Pz, bits, s_tool, obs, reward, done);
}

cudaError_t configure_warm_step(size_t smem, bool jit) {
    static size_t configured[2] = {48 * 1024, 48 * 1024};
    if (smem > configured[jit]) {
        cudaError_t e = jit ? cudaFuncSetAttribute(warm_step_jit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   int(smem))
                            : cudaFuncSetAttribute(warm_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   int(smem));
        if (e != cudaSuccess) return e;
        configured[jit] = smem;
    }
    return cudaSuccess;
}

cudaError_t launch_warm_step(const SimDev& S, const MlpDev& net, const SubstepCtl& C, const int* env_list,
                             int n_list, size_t smem, bool jit, const float* actions, float* obs, float* reward,
                             uint8_t* done, cudaStream_t st) {
    if (n_list <= 0) return cudaSuccess;
    const cudaError_t ce = configure_warm_step(smem, jit);
    if (ce != cudaSuccess) return ce;
    if (jit)
        warm_step_jit_kernel<<<n_list, kWarmThreads, smem, st>>>(S, net, C, env_list, n_list, actions, obs, reward,
                                                                 done);
    else
        warm_step_kernel<<<n_list, kWarmThreads, smem, st>>>(S, net, C, env_list, n_list, actions, obs, reward, done);
    return cudaGetLastError();
}

}  // namespace ffsrl
