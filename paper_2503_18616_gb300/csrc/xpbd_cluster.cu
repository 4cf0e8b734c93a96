// XPBD step of meshes too large for one CTA's shared memory (sm_103a):
// a thread-block cluster of CL CTAs holds one env, each CTA the positions of
// one contiguous range of part_slots slots in its shared memory, and every CTA
// reaches the others' ranges through distributed shared memory
// (ld/st.shared::cluster on addresses from mapa). The schedule splits every
// colour into CL segments by the range of the record's first vertex, so CTA r
// projects the records that mostly touch its own range; a cluster barrier
// separates colours. Arithmetic, order within colours and the per-vertex
// passes are those of the single-CTA step kernel (Algorithm 1 with the
// readings of the oracle), so results are bit-identical to it.
#include <cstdint>

#include "xpbd_device.cuh"
#include "xpbd_launch.h"
#include "xpbd_project.cuh"

namespace ffsrl {

namespace {

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(uint32_t(__cvta_generic_to_shared(p))), "r"(rank));
    return a;
}
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float4 cl_ld4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ void cl_st4(uint32_t a, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint32_t cl_ld1(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

// Positions of one env spread over the cluster: slot s lives in CTA s / P at
// row s % P of that CTA's position array.
template <int CL>
struct ClusterX {
    uint32_t base[CL];
    int P;
    __device__ __forceinline__ uint32_t addr(int s) const {
        int r = 0;
#pragma unroll
        for (int q = 1; q < CL; ++q) r += s >= q * P;
        return base[r] + uint32_t(s - r * P) * 16u;
    }
    __device__ __forceinline__ float4 ld(int s) const { return cl_ld4(addr(s)); }
    __device__ __forceinline__ void st(int s, float4 v) const { cl_st4(addr(s), v); }
};

}  // namespace

size_t cluster_smem_bytes(int part_slots) { return size_t(part_slots) * 16 + size_t(part_slots / 32) * 4; }

template <int SUB, int CL>
__global__ void __launch_bounds__(SUB, 1)
    xpbd_cluster_kernel(SimDev S, const int* __restrict__ env_list, int n_list, const float* __restrict__ actions,
                        float* __restrict__ obs, float* __restrict__ reward, uint8_t* __restrict__ done) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double s_tool[3];
    const int rank = int(cl_rank());
    const int li = blockIdx.x / CL;
    const int tid = threadIdx.x;
    if (li >= n_list) return;   // whole clusters only (the grid is n_list * CL)
    const int env = env_list ? env_list[li] : li;
    const EnvDev ed = S.envs[env];
    const MeshDev& M = S.meshes[ed.mesh];
    const int V = M.V, P = M.part_slots;
    const int n_col = M.n_ecol + M.n_tcol;
    const long long stride = S.stride;
    const int lo = rank * P, hi = min(V, lo + P);
    float4* Xl = reinterpret_cast<float4*>(smem_raw);            // own range, row s - lo
    unsigned* bits = reinterpret_cast<unsigned*>(smem_raw + size_t(P) * 16);   // own vertex range
    ClusterX<CL> X;
    X.P = P;
#pragma unroll
    for (int r = 0; r < CL; ++r) X.base[r] = cl_map(Xl, uint32_t(r));
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;
    for (int w = tid; w < P / 32; w += SUB) bits[w] = 0u;
    if (rank == 0 && tid == 0) {
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
        // Load the own slot range (its vertices are the same aligned blocks) and predict.
        const float* gx = S.x + ed.voff;
        const float* gv = S.v + ed.voff;
        // two slots per loop trip, their loads issued together
        for (int s0 = lo + tid; s0 < hi; s0 += 2 * SUB) {
            int iv[2];
            float4 xs[2];
            float vx[2], vy[2], vz[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) iv[u] = M.vert_of[s0 + u * SUB < hi ? s0 + u * SUB : s0];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = iv[u];
                xs[u] = make_float4(gx[i], gx[stride + i], gx[2 * stride + i], M.rest_w[i].w);
                vx[u] = gv[i];
                vy[u] = gv[stride + i];
                vz[u] = gv[2 * stride + i];
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int s = s0 + u * SUB;
                if (s >= hi) break;
                float4 xi = xs[u];
                Px[s] = xi.x;
                Py[s] = xi.y;
                Pz[s] = xi.z;
                if (xi.w > 0.f) {   // rounding spelled out, as in the single-CTA kernel
                    xi.x = __fmaf_rn(h, __fadd_rn(vx[u], hgx), xi.x);
                    xi.y = __fmaf_rn(h, __fadd_rn(vy[u], hgy), xi.y);
                    xi.z = __fmaf_rn(h, __fadd_rn(vz[u], hgz), xi.z);
                }
                Xl[s - lo] = xi;
            }
        }
    }
    cl_sync();   // every range loaded, the tool centre published by CTA 0
    double tool[3];
    {
        const uint32_t ta = cl_map(s_tool, 0u);
#pragma unroll
        for (int k = 0; k < 3; ++k) tool[k] = cl_ld_f64(ta + 8u * k);
    }
    const float cx = float(tool[0]), cy = float(tool[1]), cz = float(tool[2]);
    const float rad = S.radius, rad2 = __fmul_rn(rad, rad);
    const float at_d = ed.alpha_d, at_v = S.alpha_v;
    float* lam = S.lambda ? S.lambda + ed.loff : nullptr;

    // Constraint records come from L2. Each thread keeps its next record in
    // flight one loop trip ahead. (Requesting a colour's first record before
    // the previous colour's cluster barrier is slower: the barrier's release
    // semantics wait for the load.)
    auto first_rec = [&](int c) {
        const int4 sg = M.segs[c * CL + rank];
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (tid < sg.z) {
            if (c < M.n_ecol) {
                const uint2 e = __ldg(reinterpret_cast<const uint2*>(M.recs + sg.x) + tid);
                r = make_uint4(e.x, e.y, 0u, 0u);
            } else {
                r = __ldg(reinterpret_cast<const uint4*>(M.recs + sg.x) + tid);
            }
        }
        return r;
    };
    for (int sub = 0; sub < S.substeps; ++sub) {
        for (int it = 0; it < S.iterations; ++it) {
            for (int c = 0; c < n_col; ++c) {
                const int4 sg = M.segs[c * CL + rank];
                const unsigned char* base = M.recs + sg.x;
                const bool carry = lam != nullptr;
                uint4 cur = first_rec(c);
                // one iteration keeps no multipliers: loops without their loads and stores
                if (c < M.n_ecol) {
                    const uint2* rec = reinterpret_cast<const uint2*>(base);
                    for (int q = tid; q < sg.z; q += SUB) {
                        uint4 nxt = cur;
                        if (q + SUB < sg.z) {
                            const uint2 e = __ldg(rec + q + SUB);
                            nxt = make_uint4(e.x, e.y, 0u, 0u);
                        }
                        if (!carry) {
                            float l = 0.f;
                            project_edge<false>(X, make_uint2(cur.x, cur.y), at_d, M.min_len2, l);
                        } else {
                            float l = it > 0 ? lam[sg.w + q] : 0.f;
                            project_edge(X, make_uint2(cur.x, cur.y), at_d, M.min_len2, l);
                            lam[sg.w + q] = l;
                        }
                        cur = nxt;
                    }
                } else {
                    const uint4* rec = reinterpret_cast<const uint4*>(base);
                    for (int q = tid; q < sg.z; q += SUB) {
                        const uint4 nxt = (q + SUB < sg.z) ? __ldg(rec + q + SUB) : cur;
                        if (!carry) {
                            float l = 0.f;
                            project_tet<false>(X, cur, at_v, l);
                        } else {
                            float l = it > 0 ? lam[sg.w + q] : 0.f;
                            project_tet(X, cur, at_v, l);
                            lam[sg.w + q] = l;
                        }
                        cur = nxt;
                    }
                }
                cl_sync();
            }
        }
        // Collision, and except after the last substep the velocity update and
        // the next prediction, on the own range (as the single-CTA kernel).
        const bool last = sub == S.substeps - 1;
        auto vertex_pass = [&](int s, float4 xi, float px, float py, float pz) {
            if (!(xi.w > 0.f)) {
                if (!last) {
                    Px[s] = xi.x;
                    Py[s] = xi.y;
                    Pz[s] = xi.z;
                }
                return;
            }
            const float dx = __fsub_rn(xi.x, cx), dy = __fsub_rn(xi.y, cy), dz = __fsub_rn(xi.z, cz);
            const float l2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            bool moved = false;
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
                moved = true;
                if (last) {
                    const int i = M.vert_of[s] - lo;   // own vertex range is [lo, hi)
                    atomicOr(&bits[i >> 5], 1u << (i & 31));
                }
            }
            if (!last) {
                const float vx = __fmul_rn(__fsub_rn(xi.x, px), inv_h), vy = __fmul_rn(__fsub_rn(xi.y, py), inv_h),
                            vz = __fmul_rn(__fsub_rn(xi.z, pz), inv_h);
                Px[s] = xi.x;
                Py[s] = xi.y;
                Pz[s] = xi.z;
                xi.x = __fmaf_rn(h, __fadd_rn(vx, hgx), xi.x);
                xi.y = __fmaf_rn(h, __fadd_rn(vy, hgy), xi.y);
                xi.z = __fmaf_rn(h, __fadd_rn(vz, hgz), xi.z);
                moved = true;
            }
            if (moved) Xl[s - lo] = xi;
        };
        // two slots per loop trip, both slots' substep-start positions loaded first
        for (int s = lo + tid; s < hi; s += 2 * SUB) {
            const int s2 = s + SUB;
            const bool two = s2 < hi;
            const float4 x1 = Xl[s - lo];
            const float4 x2 = two ? Xl[s2 - lo] : x1;
            float p1x = 0.f, p1y = 0.f, p1z = 0.f, p2x = 0.f, p2y = 0.f, p2z = 0.f;
            if (!last) {
                p1x = Px[s];
                p1y = Py[s];
                p1z = Pz[s];
                if (two) {
                    p2x = Px[s2];
                    p2y = Py[s2];
                    p2z = Pz[s2];
                }
            }
            vertex_pass(s, x1, p1x, p1y, p1z);
            if (two) vertex_pass(s2, x2, p2x, p2y, p2z);
        }
        cl_sync();
    }
    // Write back the own range: x and v = (x - x_prev) / h in vertex order.
    float* ox = S.x + ed.voff;
    float* ov = S.v + ed.voff;
    bool bad = false;
    for (int s0 = lo + tid; s0 < hi; s0 += 2 * SUB) {   // two slots per trip, loads first
        int iv[2];
        float px[2], py[2], pz[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = s0 + u * SUB < hi ? s0 + u * SUB : s0;
            iv[u] = M.vert_of[s];
            px[u] = Px[s];
            py[u] = Py[s];
            pz[u] = Pz[s];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int s = s0 + u * SUB;
            if (s >= hi) break;
            const int i = iv[u];
            const float4 xi = Xl[s - lo];
            ox[i] = xi.x;
            ox[stride + i] = xi.y;
            ox[2 * stride + i] = xi.z;
            ov[i] = __fmul_rn(__fsub_rn(xi.x, px[u]), inv_h);
            ov[stride + i] = __fmul_rn(__fsub_rn(xi.y, py[u]), inv_h);
            ov[2 * stride + i] = __fmul_rn(__fsub_rn(xi.z, pz[u]), inv_h);
            bad |= !(isfinite(xi.x) && isfinite(xi.y) && isfinite(xi.z));
        }
    }
    if (bad) atomicOr(&S.err[env], kErrNonFinite);
    if (rank == 0) {
        // Contacts (ascending vertex ids) from every CTA's bits, observation,
        // reward and termination, read through the cluster.
        const int lane = tid & 31, warp = tid >> 5;
        if (warp == 0) {
            const int nwords = (V + 31) / 32;
            int base = 0;
            for (int w0 = 0; w0 < nwords; w0 += 32) {
                const int w = w0 + lane;
                unsigned word = 0u;
                if (w < nwords) {
                    const int r = (w * 32) / P;
                    word = cl_ld1(cl_map(bits, uint32_t(r)) + 4u * uint32_t(w - r * (P / 32)));
                }
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
                    S.contacts[ed.voff + pos++] = w * 32 + bit;
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
                    val = float(tool[j]);
                } else {
                    const int q = (j - 3) / 3, kk = (j - 3) - 3 * q;
                    const float4 xv = X.ld(M.slot_of[ids[q]]);
                    val = kk == 0 ? xv.x : (kk == 1 ? xv.y : xv.z);
                }
                o[j] = val;
            }
        }
        if (tid == 0) {
            const float4 xt = X.ld(M.slot_of[S.target[env]]);
            const double dx = tool[0] - double(xt.x), dy = tool[1] - double(xt.y), dz = tool[2] - double(xt.z);
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
    cl_sync();   // no CTA leaves while CTA 0 still reads its shared memory
}

template <int SUB, int CL>
static cudaError_t launch_cluster_one(const SimDev& S, const int* env_list, int n_list, size_t smem, cudaStream_t st,
                                      const float* a, float* o, float* r, uint8_t* d) {
    static size_t configured = 48 * 1024;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(xpbd_cluster_kernel<SUB, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    if (n_list <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(n_list) * CL, 1, 1);
    cfg.blockDim = dim3(SUB, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, xpbd_cluster_kernel<SUB, CL>, S, env_list, n_list, a, o, r, d);
}

bool cluster_config_supported(int sub, int cl) { return (sub == 512 || sub == 1024) && (cl == 2 || cl == 4); }

cudaError_t launch_cluster_step(const SimDev& S, int sub, int cl, const int* env_list, int n_list, size_t smem,
                                cudaStream_t st, const float* a, float* o, float* r, uint8_t* d) {
    if (sub == 512 && cl == 2) return launch_cluster_one<512, 2>(S, env_list, n_list, smem, st, a, o, r, d);
    if (sub == 512 && cl == 4) return launch_cluster_one<512, 4>(S, env_list, n_list, smem, st, a, o, r, d);
    if (sub == 1024 && cl == 2) return launch_cluster_one<1024, 2>(S, env_list, n_list, smem, st, a, o, r, d);
    if (sub == 1024 && cl == 4) return launch_cluster_one<1024, 4>(S, env_list, n_list, smem, st, a, o, r, d);
    return cudaErrorInvalidValue;
}

int cluster_max_active(int sub, int cl, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(cl), 1, 1);
    cfg.blockDim = dim3(unsigned(sub), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cl);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (sub == 512 && cl == 2) {
        launch_cluster_one<512, 2>(SimDev{}, nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr);
        e = cudaOccupancyMaxActiveClusters(&n, xpbd_cluster_kernel<512, 2>, &cfg);
    } else if (sub == 512 && cl == 4) {
        launch_cluster_one<512, 4>(SimDev{}, nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr);
        e = cudaOccupancyMaxActiveClusters(&n, xpbd_cluster_kernel<512, 4>, &cfg);
    } else if (sub == 1024 && cl == 2) {
        launch_cluster_one<1024, 2>(SimDev{}, nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr);
        e = cudaOccupancyMaxActiveClusters(&n, xpbd_cluster_kernel<1024, 2>, &cfg);
    } else if (sub == 1024 && cl == 4) {
        launch_cluster_one<1024, 4>(SimDev{}, nullptr, 0, smem, nullptr, nullptr, nullptr, nullptr, nullptr);
        e = cudaOccupancyMaxActiveClusters(&n, xpbd_cluster_kernel<1024, 4>, &cfg);
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace ffsrl
