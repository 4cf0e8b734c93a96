// Batched XPBD step kernels for GB300 (sm_103a).
//
// One CTA advances one environment through a whole simulation step
// (FF-SRL, arXiv 2503.18616, Algorithm 1): tool update, `substeps` substeps of
// predict -> coloured Gauss-Seidel projection of the edge-distance (Eq. 1) and
// tet-volume (Eqs. 2-3) constraints in XPBD compliance form -> sphere-tool
// collision -> velocity update, then observation, reward and termination
// (Sec. III-B, Sec. IV).
//
// Resident variant (RES = true): the env's positions live in shared memory for
// the whole step as float4 (x, y, z, inverse mass), so the 10 substeps x 55
// colour phases never touch HBM; the only HBM traffic per env-step is reading
// and writing x and v once (48 B per vertex) plus the observation. Constraint
// tables are shared by all envs of a mesh and stay in L2.
// Non-resident variant (RES = false): identical arithmetic on a float4 working
// copy in global memory (L2-resident for the CTAs in flight), for meshes whose
// state does not fit in one CTA's shared memory.
//
// Within a colour no two constraints share a vertex, so threads of the CTA
// project one colour in parallel and a __syncthreads() separates colours; the
// result equals the sequential colour-by-colour Gauss-Seidel order.
#include <cstdint>

#include "xpbd_device.cuh"
#include "xpbd_launch.h"

namespace ffsrl {

namespace {

__device__ __forceinline__ float3 sub3(float4 a, float4 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Edge-distance constraint C = |x_a - x_b| - d in XPBD form (Eq. 1 with
// compliance): dlambda = (-C - at lambda) / (w_a + w_b + at), x_a += w_a dlambda n,
// x_b -= w_b dlambda n, n = (x_a - x_b) / |x_a - x_b|.
__device__ __forceinline__ void project_edge(float4* X, uint32_t ab, float d, float at,
                                             float min_len, float& lam) {
    const int a = int(ab & 0xffffu), b = int(ab >> 16);
    float4 xa = X[a], xb = X[b];
    const float dx = xa.x - xb.x, dy = xa.y - xb.y, dz = xa.z - xb.z;
    const float len = sqrtf(dx * dx + dy * dy + dz * dz);
    const float C = len - d;
    const float denom = xa.w + xb.w + at;
    if (len < min_len || denom == 0.f) return;
    const float dl = (-C - at * lam) / denom;
    const float s = dl / len;
    const float sa = xa.w * s, sb = xb.w * s;
    xa.x += sa * dx; xa.y += sa * dy; xa.z += sa * dz;
    xb.x -= sb * dx; xb.y -= sb * dy; xb.z -= sb * dz;
    X[a] = xa;
    X[b] = xb;
    lam += dl;
}

// Tet-volume constraint C = (x_ba x x_ca) . x_da / 6 - V0 with gradients
// g_b = x_ca x x_da / 6, g_c = x_da x x_ba / 6, g_d = x_ba x x_ca / 6,
// g_a = -(g_b + g_c + g_d) (the consistent reading of Eq. 2), scaled as in
// Eq. 3 with inverse masses and compliance: dlambda = (-C - at lambda) /
// (sum w_i |g_i|^2 + at), x_i += w_i dlambda g_i.
__device__ __forceinline__ void project_tet(float4* X, uint2 q, float V0, float at, float& lam) {
    const int a = int(q.x & 0xffffu), b = int(q.x >> 16);
    const int c = int(q.y & 0xffffu), d = int(q.y >> 16);
    float4 xa = X[a], xb = X[b], xc = X[c], xd = X[d];
    const float3 ba = sub3(xb, xa), ca = sub3(xc, xa), da = sub3(xd, xa);
    const float3 g1 = cross3(ca, da), g2 = cross3(da, ba), g3 = cross3(ba, ca);  // 6 x gradient
    const float3 g0 = make_float3(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    const float C = dot3(g3, da) * (1.0f / 6.0f) - V0;
    const float sw = xa.w * dot3(g0, g0) + xb.w * dot3(g1, g1) + xc.w * dot3(g2, g2) + xd.w * dot3(g3, g3);
    const float denom = sw * (1.0f / 36.0f) + at;
    if (denom == 0.f) return;
    const float dl = (-C - at * lam) / denom;
    const float s = dl * (1.0f / 6.0f);
    const float sa = xa.w * s, sb = xb.w * s, sc = xc.w * s, sd = xd.w * s;
    xa.x += sa * g0.x; xa.y += sa * g0.y; xa.z += sa * g0.z;
    xb.x += sb * g1.x; xb.y += sb * g1.y; xb.z += sb * g1.z;
    xc.x += sc * g2.x; xc.y += sc * g2.y; xc.z += sc * g2.z;
    xd.x += sd * g3.x; xd.y += sd * g3.y; xd.z += sd * g3.z;
    X[a] = xa;
    X[b] = xb;
    X[c] = xc;
    X[d] = xd;
    lam += dl;
}

}  // namespace

size_t resident_smem_bytes(int Vp) {
    return size_t(Vp) * sizeof(float4) + 3 * size_t(Vp) * sizeof(float) + size_t(Vp / 32) * 4;
}
size_t streaming_smem_bytes(int Vp) { return size_t(Vp / 32) * 4; }

template <int BLOCK, bool RES>
__global__ void __launch_bounds__(BLOCK) xpbd_step_kernel(SimDev S, const int* __restrict__ env_list,
                                                          const float* __restrict__ actions,
                                                          float* __restrict__ obs,
                                                          float* __restrict__ reward,
                                                          uint8_t* __restrict__ done) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int env = env_list ? env_list[blockIdx.x] : int(blockIdx.x);
    const int tid = threadIdx.x;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const int V = M.V, Vp = M.Vp;
    const long long stride = S.stride;

    float4* X;
    float *Px, *Py, *Pz;
    unsigned* bits;
    if constexpr (RES) {
        X = reinterpret_cast<float4*>(smem_raw);
        Px = reinterpret_cast<float*>(X + Vp);
        Py = Px + Vp;
        Pz = Py + Vp;
        bits = reinterpret_cast<unsigned*>(Pz + Vp);
    } else {
        X = S.xg + ed.voff;
        Px = S.pg + ed.voff;
        Py = Px + stride;
        Pz = Py + stride;
        bits = reinterpret_cast<unsigned*>(smem_raw);
    }
    __shared__ double s_tool[3];

    // Tool update once per step (Algorithm 1, "evaluate instrument state"):
    // c <- clamp(c + scale * a) with a from the caller or from the env's
    // counter-based stream at its current step count.
    if (tid == 0) {
        const unsigned long long t = (unsigned long long)S.t_step[env];
        const unsigned long long st = env_stream(S.seed[env], (unsigned long long)env, 0u);
        for (int k = 0; k < 3; ++k) {
            const double a = actions ? (double)actions[3 * env + k] : to_unit_pm1(splitmix64_nth(st, 3ull * t + k));
            // rounded product, then rounded sum (no fused multiply-add), so the
            // float64 tool position is reproducible bit for bit
            double c = __dadd_rn(S.tool[3 * env + k], __dmul_rn(S.action_scale, a));
            c = c < M.box_lo[k] ? M.box_lo[k] : c;
            c = c > M.box_hi[k] ? M.box_hi[k] : c;
            S.tool[3 * env + k] = c;
            s_tool[k] = c;
        }
    }

    const float h = S.h;
    const float* gx_ = S.x + ed.voff;
    const float* gy_ = gx_ + stride;
    const float* gz_ = gy_ + stride;
    const float* gvx = S.v + ed.voff;
    const float* gvy = gvx + stride;
    const float* gvz = gvy + stride;

    // Load the state and predict for the first substep (Algorithm 1:
    // v~ = v + h g, x~ = x + h v~ for free vertices).
    for (int i = tid; i < V; i += BLOCK) {
        float4 xi = make_float4(gx_[i], gy_[i], gz_[i], M.rest_w[i].w);
        Px[i] = xi.x;
        Py[i] = xi.y;
        Pz[i] = xi.z;
        if (xi.w > 0.f) {
            const float vx = gvx[i] + h * S.gx, vy = gvy[i] + h * S.gy, vz = gvz[i] + h * S.gz;
            xi.x += h * vx;
            xi.y += h * vy;
            xi.z += h * vz;
        }
        X[i] = xi;
    }
    for (int w = tid; w < Vp / 32; w += BLOCK) bits[w] = 0u;
    __syncthreads();
    const float cx = float(s_tool[0]), cy = float(s_tool[1]), cz = float(s_tool[2]);
    const float r = S.radius;
    const float at_d = ed.alpha_d, at_v = S.alpha_v;
    const int E = M.E;
    float* lam_e = S.lambda ? S.lambda + ed.loff : nullptr;
    float* lam_t = lam_e ? lam_e + E : nullptr;

    for (int sub = 0; sub < S.substeps; ++sub) {
        if (sub > 0) {
            // velocity update of the previous substep, v = (x - x_prev) / h,
            // fused with this substep's prediction.
            for (int i = tid; i < V; i += BLOCK) {
                float4 xi = X[i];
                const float vx = (xi.x - Px[i]) / h, vy = (xi.y - Py[i]) / h, vz = (xi.z - Pz[i]) / h;
                Px[i] = xi.x;
                Py[i] = xi.y;
                Pz[i] = xi.z;
                if (xi.w > 0.f) {
                    xi.x += h * (vx + h * S.gx);
                    xi.y += h * (vy + h * S.gy);
                    xi.z += h * (vz + h * S.gz);
                    X[i] = xi;
                }
            }
            __syncthreads();
        }
        for (int it = 0; it < S.iterations; ++it) {
            const bool carry = lam_e != nullptr;
            for (int col = 0; col < M.n_ecol; ++col) {
                const int beg = M.ecol_off[col], end = M.ecol_off[col + 1];
                for (int q = beg + tid; q < end; q += BLOCK) {
                    float lam = (carry && it > 0) ? lam_e[q] : 0.f;
                    project_edge(X, __ldg(M.edge_ab + q), __ldg(M.edge_d + q), at_d, M.min_len, lam);
                    if (carry) lam_e[q] = lam;
                }
                __syncthreads();
            }
            for (int col = 0; col < M.n_tcol; ++col) {
                const int beg = M.tcol_off[col], end = M.tcol_off[col + 1];
                for (int q = beg + tid; q < end; q += BLOCK) {
                    float lam = (carry && it > 0) ? lam_t[q] : 0.f;
                    project_tet(X, __ldg(M.tet_abcd + q), __ldg(M.tet_V0 + q), at_v, lam);
                    if (carry) lam_t[q] = lam;
                }
                __syncthreads();
            }
        }
        // Sphere-tool collision (Sec. III-A "Collisions"): a free vertex
        // closer than r to the centre is moved onto the sphere along the
        // centre-to-vertex direction (straight up if it sits on the centre).
        const bool last = sub == S.substeps - 1;
        for (int i = tid; i < V; i += BLOCK) {
            float4 xi = X[i];
            if (xi.w > 0.f) {
                const float dx = xi.x - cx, dy = xi.y - cy, dz = xi.z - cz;
                const float len = sqrtf(dx * dx + dy * dy + dz * dz);
                if (len < r) {
                    if (len > 0.f) {
                        xi.x = cx + r * (dx / len);
                        xi.y = cy + r * (dy / len);
                        xi.z = cz + r * (dz / len);
                    } else {
                        xi.x = cx;
                        xi.y = cy;
                        xi.z = cz + r;
                    }
                    X[i] = xi;
                    if (last) atomicOr(&bits[i >> 5], 1u << (i & 31));
                }
            }
        }
    }
    __syncthreads();

    // Write back x and v = (x - x_prev) / h; flag non-finite positions.
    float* ox = S.x + ed.voff;
    float* oy = ox + stride;
    float* oz = oy + stride;
    float* ovx = S.v + ed.voff;
    float* ovy = ovx + stride;
    float* ovz = ovy + stride;
    int bad = 0;
    for (int i = tid; i < V; i += BLOCK) {
        const float4 xi = X[i];
        ox[i] = xi.x;
        oy[i] = xi.y;
        oz[i] = xi.z;
        ovx[i] = (xi.x - Px[i]) / h;
        ovy[i] = (xi.y - Py[i]) / h;
        ovz[i] = (xi.z - Pz[i]) / h;
        bad |= !(isfinite(xi.x) && isfinite(xi.y) && isfinite(xi.z));
    }
    bad = __syncthreads_or(bad);

    // Contact list of the last substep, ascending vertex ids (warp 0).
    const int lane = tid & 31, warp = tid >> 5;
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

    // Observation: tool centre, then the sampled top-face vertices (Sec. IV).
    if (obs) {
        float* o = obs + (long long)env * S.obs_dim;
        const int* ids = S.obs_ids + (long long)env * S.n_obs;
        for (int j = tid; j < S.obs_dim; j += BLOCK) {
            float val;
            if (j < 3) {
                val = float(s_tool[j]);
            } else {
                const int q = (j - 3) / 3, k = (j - 3) - 3 * q;
                const float4 xv = X[ids[q]];
                val = k == 0 ? xv.x : (k == 1 ? xv.y : xv.z);
            }
            o[j] = val;
        }
    }
    // Reward R = w_l l + w_d (l - l_prev) + w_s s and termination (Sec. IV, Sec. III-B).
    if (tid == 0) {
        const float4 xt = X[S.target[env]];
        const double dx = s_tool[0] - double(xt.x), dy = s_tool[1] - double(xt.y), dz = s_tool[2] - double(xt.z);
        const double l = sqrt(dx * dx + dy * dy + dz * dz);
        const int succ = l < S.success_dist;
        const double R = S.w_l * l + S.w_d * (l - double(S.l_prev[env])) + S.w_s * double(succ);
        S.l_prev[env] = float(l);
        const int t = S.t_step[env] + 1;
        S.t_step[env] = t;
        if (reward) reward[env] = float(R);
        if (done) done[env] = uint8_t(((S.max_steps > 0 && t >= S.max_steps) || succ) ? 1 : 0);
        if (bad) S.err[env] |= 1;
    }
}

// Episode reset (Sec. III-B): rest positions, zero velocities, tool at its
// start, fresh observed vertices (Floyd's sampling without replacement from
// the top face, sorted) and target vertex from the env's counter-based streams.
__global__ void reset_kernel(SimDev S, const uint8_t* __restrict__ mask, unsigned long long seed) {
    const int env = blockIdx.x;
    if (mask && !mask[env]) return;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const long long stride = S.stride;
    for (int i = threadIdx.x; i < M.V; i += blockDim.x) {
        const float4 r = M.rest_w[i];
        S.x[ed.voff + i] = r.x;
        S.x[stride + ed.voff + i] = r.y;
        S.x[2 * stride + ed.voff + i] = r.z;
        S.v[ed.voff + i] = 0.f;
        S.v[stride + ed.voff + i] = 0.f;
        S.v[2 * stride + ed.voff + i] = 0.f;
    }
    if (threadIdx.x == 0) {
        int* ids = S.obs_ids + (long long)env * S.n_obs;
        const unsigned long long st = env_stream(seed, (unsigned long long)env, 1u);
        const int n = M.n_top, k = S.n_obs;
        int m = 0;
        for (int j = n - k; j < n; ++j) {
            const int t = int(splitmix64_nth(st, (unsigned long long)j) % (unsigned long long)(j + 1));
            bool taken = false;
            for (int q = 0; q < m; ++q) taken |= (ids[q] == t);
            ids[m++] = taken ? j : t;
        }
        for (int a = 1; a < m; ++a) {
            const int key = ids[a];
            int b = a - 1;
            while (b >= 0 && ids[b] > key) { ids[b + 1] = ids[b]; --b; }
            ids[b + 1] = key;
        }
        for (int q = 0; q < m; ++q) ids[q] = M.top[ids[q]];
        const int tgt = M.top[splitmix64_nth(env_stream(seed, (unsigned long long)env, 2u), 0ull) %
                              (unsigned long long)n];
        S.target[env] = tgt;
        const float4 rt = M.rest_w[tgt];
        double l2 = 0;
        for (int kk = 0; kk < 3; ++kk) {
            S.tool[3 * env + kk] = M.tool_start[kk];
            const double dk = M.tool_start[kk] - double(kk == 0 ? rt.x : (kk == 1 ? rt.y : rt.z));
            l2 += dk * dk;
        }
        S.l_prev[env] = float(sqrt(l2));
        S.t_step[env] = 0;
        S.seed[env] = seed;
        S.n_contacts[env] = 0;
    }
}

// Packed [rows][3] <-> padded structure-of-arrays copies (state access).
__global__ void pack_state_kernel(SimDev S, const int* __restrict__ pstart, float* __restrict__ xo,
                                  float* __restrict__ vo) {
    const int env = blockIdx.x;
    const EnvDev ed = S.envs[env];
    const int V = S.meshes[ed.mesh].V;
    const long long p0 = pstart[env];
    for (int i = threadIdx.x; i < V; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            if (xo) xo[3 * (p0 + i) + k] = S.x[k * S.stride + ed.voff + i];
            if (vo) vo[3 * (p0 + i) + k] = S.v[k * S.stride + ed.voff + i];
        }
}

__global__ void unpack_state_kernel(SimDev S, const int* __restrict__ pstart, const float* __restrict__ xi,
                                    const float* __restrict__ vi) {
    const int env = blockIdx.x;
    const EnvDev ed = S.envs[env];
    const int V = S.meshes[ed.mesh].V;
    const long long p0 = pstart[env];
    for (int i = threadIdx.x; i < V; i += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            if (xi) S.x[k * S.stride + ed.voff + i] = xi[3 * (p0 + i) + k];
            if (vi) S.v[k * S.stride + ed.voff + i] = vi[3 * (p0 + i) + k];
        }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <int BLOCK, bool RES>
static cudaError_t launch_one(const SimDev& S, const int* env_list, int n_blocks, size_t smem,
                              cudaStream_t st, const float* actions, float* obs, float* reward, uint8_t* done) {
    // Raise the kernel's dynamic shared-memory limit to what this launch needs
    // (the limit plus the kernel's static shared memory must stay within the
    // device's per-block opt-in maximum).
    static size_t configured = 48 * 1024;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(xpbd_step_kernel<BLOCK, RES>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    xpbd_step_kernel<BLOCK, RES><<<n_blocks, BLOCK, smem, st>>>(S, env_list, actions, obs, reward, done);
    return cudaGetLastError();
}

template <bool RES>
static cudaError_t launch_block(int block, const SimDev& S, const int* env_list, int n_blocks, size_t smem,
                                cudaStream_t st, const float* a, float* o, float* r, uint8_t* d) {
    switch (block) {
    case 128: return launch_one<128, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    case 256: return launch_one<256, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    case 384: return launch_one<384, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    case 512: return launch_one<512, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    case 768: return launch_one<768, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    case 1024: return launch_one<1024, RES>(S, env_list, n_blocks, smem, st, a, o, r, d);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(const SimDev& S, bool resident, int block, const int* env_list, int n_blocks,
                        size_t smem_bytes, cudaStream_t stream, const float* actions, float* obs,
                        float* reward, uint8_t* done) {
    if (n_blocks <= 0) return cudaSuccess;
    return resident ? launch_block<true>(block, S, env_list, n_blocks, smem_bytes, stream, actions, obs, reward, done)
                    : launch_block<false>(block, S, env_list, n_blocks, smem_bytes, stream, actions, obs, reward, done);
}

cudaError_t launch_reset(const SimDev& S, const uint8_t* mask, unsigned long long seed, cudaStream_t st) {
    reset_kernel<<<S.n_env, 256, 0, st>>>(S, mask, seed);
    return cudaGetLastError();
}

cudaError_t launch_pack(const SimDev& S, const int* pstart, float* x, float* v, cudaStream_t st) {
    pack_state_kernel<<<S.n_env, 256, 0, st>>>(S, pstart, x, v);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const SimDev& S, const int* pstart, const float* x, const float* v, cudaStream_t st) {
    unpack_state_kernel<<<S.n_env, 256, 0, st>>>(S, pstart, x, v);
    return cudaGetLastError();
}

}  // namespace ffsrl
