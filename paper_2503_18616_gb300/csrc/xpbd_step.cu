// Batched XPBD step kernels for GB300 (sm_103a).
//
// One CTA advances one environment through a whole simulation step
// (FF-SRL, arXiv 2503.18616, Algorithm 1): tool update, `substeps` substeps of
// predict -> coloured Gauss-Seidel projection of the edge-distance (Eq. 1) and
// tet-volume (Eqs. 2-3) constraints in XPBD compliance form -> sphere-tool
// collision -> velocity update, then observation, reward and termination
// (Sec. III-B, Sec. IV).
//
// Resident variant (RES): the env's positions live in shared memory for the
// whole step as float4 (x, y, z, inverse mass) in slot order, so the
// substeps x colours phases never touch HBM; per env-step the HBM traffic is
// x and v read and written once (48 B per vertex) plus the observation.
// Non-resident variant: the same arithmetic on a float4 working copy in
// global memory (L2-resident while its CTA runs), for meshes too large for one
// CTA's shared memory.
// Ring variant (RING): the records of the next colour are copied from the
// L2-resident constraint stream into a shared-memory double buffer by the
// Tensor Memory Accelerator (cp.async.bulk with an mbarrier) while the current
// colour is projected, so no thread waits on L2 for constraint records.
//
// Within a colour no two constraints share a vertex, so the CTA's threads
// project one colour in parallel and a barrier separates colours; the result
// equals the sequential colour-by-colour Gauss-Seidel order.
#include <cstdint>
#include <type_traits>

#include "xpbd_device.cuh"
#include "xpbd_grasper.cuh"
#include "xpbd_launch.h"
#include "xpbd_project.cuh"

namespace ffsrl {

namespace {

// ---- mbarrier and bulk-copy helpers (PTX, sm_90+) ---------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return uint32_t(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_addr(bar)),
        "r"(bytes)
        : "memory");
}
// Bulk copy global -> this CTA's shared memory; completion counted on `bar`.
// dst, src and bytes are multiples of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of parity `parity` to complete, giving up after a fixed
// number of polls (each poll may suspend the thread briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__host__ __device__ __forceinline__ size_t align128(size_t b) { return (b + 127) / 128 * 128; }

// Dynamic shared-memory layout of a CTA holding `envs` envs:
// [X of each env (resident only)] [ring (2 stages, shared)] [segment table] [contact bits of each env]
struct SmemLayout {
    size_t x_off, ring_off, seg_off, bits_off, total;
    __host__ __device__ SmemLayout(int Vp, bool res, bool ring, int ring_bytes, int n_seg, int envs) {
        x_off = 0;
        ring_off = align128(res ? size_t(envs) * Vp * 16 : 0);
        seg_off = align128(ring_off + (ring ? 2 * size_t(ring_bytes) : 0));
        bits_off = align128(seg_off + size_t(n_seg) * 16);
        total = bits_off + size_t(envs) * (Vp / 32) * 4;
    }
};

}  // namespace

size_t step_smem_bytes(int Vp, bool resident, bool ring, int ring_bytes, int n_seg, int envs) {
    return SmemLayout(Vp, resident, ring, ring_bytes, n_seg, envs).total;
}

// CTAs per SM the register allocation targets for each block size (about 85
// registers per thread at 768 threads per SM, 64 at 1024).
constexpr int min_ctas_per_sm(int block) {
    return block <= 128 ? 6 : block <= 256 ? 3 : block <= 512 ? 2 : 1;
}

// One CTA advances ENVS environments of the same mesh, SUB threads each; the
// envs share the constraint ring and the CTA's barriers.
template <int SUB, int ENVS, bool RES, bool RING, int OCC = 0>
__global__ void __launch_bounds__(SUB * ENVS, OCC ? OCC : min_ctas_per_sm(SUB * ENVS))
    xpbd_step_kernel(SimDev S, const int* __restrict__ env_list, int n_list, const float* __restrict__ actions,
                     float* __restrict__ obs, float* __restrict__ reward, uint8_t* __restrict__ done) {
    constexpr int BLOCK = SUB * ENVS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ double s_tool[ENVS][3];

    const int tid = threadIdx.x;
    const int el = ENVS == 1 ? 0 : tid / SUB;   // env slot of this thread in the CTA
    const int st = ENVS == 1 ? tid : tid % SUB; // thread index inside the env's subgroup
    const int li = blockIdx.x * ENVS + el;
    const bool active = li < n_list;
    const int env = active ? (env_list ? env_list[li] : li) : 0;
    const EnvDev ed = S.envs[env];
    const int mesh = S.envs[env_list ? env_list[blockIdx.x * ENVS] : blockIdx.x * ENVS].mesh;
    const MeshDev M = S.meshes[mesh];
    const int V = M.V, Vp = M.Vp, n_seg = M.n_seg, n_ecol = M.n_ecol;
    const long long stride = S.stride;
    const SmemLayout L(Vp, RES, RING, M.ring_bytes, n_seg, ENVS);

    float4* X = RES ? reinterpret_cast<float4*>(smem_raw + L.x_off) + size_t(el) * Vp : S.xg + ed.voff;
    // The four-CTA build reads the record stream whose slot fields are byte
    // offsets (its meshes have at most 4096 slots): no shift per vertex access.
    constexpr bool BYTES = OCC == 4 && RES;
    using Acc = typename std::conditional<BYTES, SmemXB, SmemX>::type;
    const Acc XA{reinterpret_cast<decltype(Acc::p)>(X)};
    const unsigned char* recs = BYTES ? M.recs16 : M.recs;
    unsigned char* ring = smem_raw + L.ring_off;
    int4* segs = reinterpret_cast<int4*>(smem_raw + L.seg_off);
    unsigned* bits = reinterpret_cast<unsigned*>(smem_raw + L.bits_off) + size_t(el) * (Vp / 32);
    float* Px = S.pg + ed.voff;
    float* Py = Px + stride;
    float* Pz = Py + stride;

    const int K = S.substeps * S.iterations * n_seg;  // colour phases in this step
    for (int c = tid; c < n_seg; c += BLOCK) segs[c] = M.segs[c];
    for (int w = st; w < Vp / 32; w += SUB) bits[w] = 0u;
    if (RING && tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    if (st == 0 && active) {
        // Tool update once per step (Algorithm 1, "evaluate instrument
        // state"): c <- clamp(c + scale * a), a from the caller or from the
        // env's counter-based stream at its step count. Rounded product then
        // rounded sum, so the float64 tool position is reproducible.
        const unsigned long long t = (unsigned long long)S.t_step[env];
        const unsigned long long rs = env_stream(S.seed[env], ed.gid, 0u);
        for (int k = 0; k < 3; ++k) {
            const double a = actions ? (double)actions[3 * env + k] : to_unit_pm1(splitmix64_nth(rs, 3ull * t + k));
            double c = __dadd_rn(S.tool[3 * env + k], __dmul_rn(S.action_scale, a));
            c = c < M.box_lo[k] ? M.box_lo[k] : c;
            c = c > M.box_hi[k] ? M.box_hi[k] : c;
            S.tool[3 * env + k] = c;
            s_tool[el][k] = c;
        }
    }
    __syncthreads();
    // Prefetch the first colour while the state loads.
    if (RING && tid == 0 && K > 0) {
        const int4 sg = segs[0];
        mbar_expect_tx(&mbar[0], uint32_t(sg.y));
        bulk_copy_g2s(ring, recs + sg.x, uint32_t(sg.y), &mbar[0]);
    }

    const float h = S.h, inv_h = S.inv_h;
    const float hgx = __fmul_rn(h, S.gx), hgy = __fmul_rn(h, S.gy), hgz = __fmul_rn(h, S.gz);
    if (active) {
        // Load the state (vertex order, coalesced) into slot order and predict
        // for the first substep (Algorithm 1: v~ = v + h g, x~ = x + h v~).
        const float* gx = S.x + ed.voff;
        const float* gv = S.v + ed.voff;
        constexpr int NL = 4;   // vertices per loop trip, their loads issued together
        for (int i0 = st; i0 < V; i0 += NL * SUB) {
            int sl[NL];
            float4 xs[NL];
            float vx[NL], vy[NL], vz[NL];
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int i = i0 + u * SUB < V ? i0 + u * SUB : i0;
                sl[u] = M.slot_of[i];
                xs[u] = make_float4(gx[i], gx[stride + i], gx[2 * stride + i], M.rest_w[i].w);
                vx[u] = gv[i];
                vy[u] = gv[stride + i];
                vz[u] = gv[2 * stride + i];
            }
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                if (i0 + u * SUB >= V) break;
                const int s = sl[u];
                float4 xi = xs[u];
                Px[s] = xi.x;
                Py[s] = xi.y;
                Pz[s] = xi.z;
                if (xi.w > 0.f) {   // rounding spelled out: the same bits in every kernel instantiation
                    xi.x = __fmaf_rn(h, __fadd_rn(vx[u], hgx), xi.x);
                    xi.y = __fmaf_rn(h, __fadd_rn(vy[u], hgy), xi.y);
                    xi.z = __fmaf_rn(h, __fadd_rn(vz[u], hgz), xi.z);
                }
                X[s] = xi;
            }
        }
    }
    __syncthreads();

    const float cx = float(s_tool[el][0]), cy = float(s_tool[el][1]), cz = float(s_tool[el][2]);
    const bool grasper = S.tool_model == 1;
    const float r = grasper ? 0.f : S.radius, r2 = __fmul_rn(r, r);   // the grasper replaces the sphere
    // Grasper: capsules, dragging point and grasp state, once per env and
    // step (the tool holds still through the step), in shared memory.
    __shared__ Capsules s_caps[ENVS];
    __shared__ float s_drag[ENVS][4];              // dragging point, grasp distance
    __shared__ int s_grasp[ENVS];                  // grasped slot or -1
    __shared__ unsigned long long s_key[ENVS];     // (distance bits, vertex) of the nearest candidate
    const float closed = 3.0f * 3.14159265f / 180.0f;   // clamps below 3 degrees grasp
    if (grasper) {
        if (st == 0 && active) {
            const float angle = S.clamp_angle[env];
            grasper_capsules(S, M, s_tool[el], S.clamp_cs[env], s_caps[el]);
            const float3 g = grasper_drag_point(S, M, s_tool[el]);
            s_drag[el][0] = g.x;
            s_drag[el][1] = g.y;
            s_drag[el][2] = g.z;
            s_key[el] = ~0ull;
            if (!(angle < closed)) S.grasp_v[env] = -1;   // open clamps release
        }
        __syncthreads();
        // Closed clamps without a grasp take the free vertex nearest to the
        // dragging point within the grasp radius (positions at the step's
        // start; ties: the lower vertex id).
        if (active && S.clamp_angle[env] < closed && S.grasp_v[env] < 0) {
            const float gx0 = s_drag[el][0], gy0 = s_drag[el][1], gz0 = s_drag[el][2];
            const float* px = S.x + ed.voff;
            unsigned long long best = ~0ull;
            for (int i = st; i < V; i += SUB) {
                if (!(M.rest_w[i].w > 0.f)) continue;
                const float ddx = __fsub_rn(px[i], gx0), ddy = __fsub_rn(px[stride + i], gy0),
                            ddz = __fsub_rn(px[2 * stride + i], gz0);
                const float d = sqrtf(__fadd_rn(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)), __fmul_rn(ddz, ddz)));
                if (d < S.grasp_radius) {
                    const unsigned long long key = (static_cast<unsigned long long>(__float_as_uint(d)) << 32) | unsigned(i);
                    best = key < best ? key : best;
                }
            }
            if (best != ~0ull) atomicMin(&s_key[el], best);
        }
        __syncthreads();
        if (st == 0 && active) {
            if (s_key[el] != ~0ull) {
                S.grasp_v[env] = int(s_key[el] & 0xffffffffull);
                S.grasp_d0[env] = __uint_as_float(unsigned(s_key[el] >> 32));
            }
            const int gv = S.grasp_v[env];
            s_grasp[el] = gv >= 0 ? int(M.slot_of[gv]) : -1;
            s_drag[el][3] = S.grasp_d0[env];
        }
        __syncthreads();
    }
    const float tiny_len = sqrtf(M.min_len2);   // 1e-12 x extent: the axis crosses the face
    const float at_d = ed.alpha_d, at_v = S.alpha_v;
    float* lam = S.lambda ? S.lambda + ed.loff : nullptr;
    int k = 0;
    bool failed = false;

    for (int sub = 0; sub < S.substeps && !failed; ++sub) {
        for (int it = 0; it < S.iterations && !failed; ++it) {
            for (int c = 0; c < n_seg; ++c, ++k) {
                const int4 sg = segs[c];
                const unsigned char* base = recs + sg.x;
                bool ok = true;
                if (RING) {
                    if (tid == 0 && k + 1 < K) {
                        // The other stage was read during colour k-1, which
                        // every thread finished before the last barrier.
                        const int4 nx = segs[(c + 1 == n_seg) ? 0 : c + 1];
                        uint64_t* b = &mbar[(k + 1) & 1];
                        mbar_expect_tx(b, uint32_t(nx.y));
                        bulk_copy_g2s(ring + ((k + 1) & 1) * M.ring_bytes, recs + nx.x, uint32_t(nx.y), b);
                    }
                    ok = mbar_wait_bounded(&mbar[k & 1], uint32_t((k >> 1) & 1));
                    base = ring + (k & 1) * M.ring_bytes;
                }
                const bool carry = lam != nullptr;
                if (ok && active) {
                    const bool lin = carry && it > 0;
                    // one iteration (no multipliers kept): loops without the
                    // multiplier loads and stores, with lambda = 0 as the
                    // carried loops start from
                    if (c < n_ecol) {
                        const uint2* rec = reinterpret_cast<const uint2*>(base);
                        if (!carry) {
                            for (int q = st; q < sg.z; q += SUB) {
                                float l = 0.f;
                                project_edge<false>(XA, rec[q], at_d, M.min_len2, l);
                            }
                        } else {
                            for (int q = st; q < sg.z; q += SUB) {
                                float l = lin ? lam[sg.w + q] : 0.f;
                                project_edge(XA, rec[q], at_d, M.min_len2, l);
                                lam[sg.w + q] = l;
                            }
                        }
                    } else if (c < M.n_dseg) {
                        const uint4* rec = reinterpret_cast<const uint4*>(base);
                        if (!carry) {
                            for (int q = st; q < sg.z; q += SUB) {
                                float l = 0.f;
                                project_tet<false>(XA, rec[q], at_v, l);
                            }
                        } else {
                            for (int q = st; q < sg.z; q += SUB) {
                                float l = lin ? lam[sg.w + q] : 0.f;
                                project_tet(XA, rec[q], at_v, l);
                                lam[sg.w + q] = l;
                            }
                        }
                    } else {
                        // tissue connections, after the volume colours
                        const uint4* rec = reinterpret_cast<const uint4*>(base);
                        for (int q = st; q < sg.z; q += SUB) {
                            float l = (carry && it > 0) ? lam[sg.w + q] : 0.f;
                            project_conn(XA, rec[q], at_d, M.min_len2, l);
                            if (carry) lam[sg.w + q] = l;
                        }
                    }
                }
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
            }
        }
        if (failed) break;
        const bool last = sub == S.substeps - 1;
        if (grasper) {
            // Dragging constraint of the grasped vertex, then the grasper
            // against the surface faces, colour by colour (faces of one
            // colour share no vertex).
            if (st == 0 && active && s_grasp[el] >= 0)
                grasper_drag(X, s_grasp[el], make_float3(s_drag[el][0], s_drag[el][1], s_drag[el][2]), s_drag[el][3]);
            __syncthreads();
            for (int fc = 0; fc < M.n_fcol; ++fc) {
                if (active)
                    for (int q = M.fcol_off[fc] + st; q < M.fcol_off[fc + 1]; q += SUB)
                        grasper_face(X, M.frec[q], s_caps[el], tiny_len, last ? bits : nullptr, M.vert_of);
                __syncthreads();
            }
        }
        // Sphere-tool collision (Sec. III-A "Collisions"): a free vertex
        // closer than r to the centre moves onto the sphere along the
        // centre-to-vertex direction (straight up if it sits on the centre).
        // Except after the last substep, the same pass performs the velocity
        // update v = (x - x_prev) / h and the next substep's prediction.
        // Several slots per loop trip, all their substep-start positions
        // loaded before any is used (the global loads of one trip overlap).
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
            if (l2 < r2) {
                const float len = sqrtf(l2);
                if (len > 0.f) {
                    const float f = __fdividef(r, len);
                    xi.x = __fmaf_rn(f, dx, cx);
                    xi.y = __fmaf_rn(f, dy, cy);
                    xi.z = __fmaf_rn(f, dz, cz);
                } else {
                    xi.x = cx;
                    xi.y = cy;
                    xi.z = __fadd_rn(cz, r);
                }
                moved = true;
                if (last) {
                    const int i = M.vert_of[s];
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
            if (moved) X[s] = xi;
        };
        if (active) {
            constexpr int NV = 4;   // slots per loop trip
            for (int s0 = st; s0 < V; s0 += NV * SUB) {
                float4 xs[NV];
                float px[NV], py[NV], pz[NV];
#pragma unroll
                for (int u = 0; u < NV; ++u) {
                    const int s = s0 + u * SUB;
                    xs[u] = s < V ? X[s] : make_float4(0.f, 0.f, 0.f, 0.f);
                    px[u] = py[u] = pz[u] = 0.f;
                    if (!last && s < V) {
                        px[u] = Px[s];
                        py[u] = Py[s];
                        pz[u] = Pz[s];
                    }
                }
#pragma unroll
                for (int u = 0; u < NV; ++u)
                    if (s0 + u * SUB < V) vertex_pass(s0 + u * SUB, xs[u], px[u], py[u], pz[u]);
            }
        }
        __syncthreads();
    }
    if (failed) {
        // A constraint copy did not arrive: drain the copy that may still be
        // in flight (bounded), flag the envs and leave their state untouched.
        if (tid == 0 && RING && k + 1 < K) mbar_wait_bounded(&mbar[(k + 1) & 1], uint32_t(((k + 1) >> 1) & 1));
        if (st == 0 && active) atomicOr(&S.err[env], kErrTimeout);
        return;
    }
    if (!active) return;  // no barrier below this point

    // Write back x and v = (x - x_prev) / h in vertex order; flag non-finite positions.
    float* ox = S.x + ed.voff;
    float* ov = S.v + ed.voff;
    bool bad = false;
    constexpr int NW = 4;   // vertices per loop trip, their loads issued together
    for (int i0 = st; i0 < V; i0 += NW * SUB) {
        int sl[NW];
#pragma unroll
        for (int u = 0; u < NW; ++u) sl[u] = i0 + u * SUB < V ? int(M.slot_of[i0 + u * SUB]) : 0;
        float4 xs[NW];
        float px[NW], py[NW], pz[NW];
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            xs[u] = X[sl[u]];
            px[u] = Px[sl[u]];
            py[u] = Py[sl[u]];
            pz[u] = Pz[sl[u]];
        }
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int i = i0 + u * SUB;
            if (i >= V) break;
            const float4 xi = xs[u];
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

    // Contact list of the last substep, ascending vertex ids (first warp of the env).
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

    // Observation: tool centre, then the sampled top-face vertices (Sec. IV).
    if (obs) {
        float* o = obs + (long long)env * S.obs_dim;
        const int* ids = S.obs_ids + (long long)env * S.n_obs;
        for (int j = st; j < S.obs_dim; j += SUB) {
            float val;
            if (j < 3) {
                val = float(s_tool[el][j]);
            } else {
                const int q = (j - 3) / 3, kk = (j - 3) - 3 * q;
                const float4 xv = X[M.slot_of[ids[q]]];
                val = kk == 0 ? xv.x : (kk == 1 ? xv.y : xv.z);
            }
            o[j] = val;
        }
    }
    // Reward R = w_l l + w_d (l - l_prev) + w_s s and termination (Sec. IV, Sec. III-B).
    if (st == 0) {
        const float4 xt = X[M.slot_of[S.target[env]]];
        const double dx = s_tool[el][0] - double(xt.x), dy = s_tool[el][1] - double(xt.y),
                     dz = s_tool[el][2] - double(xt.z);
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

// Episode reset (Sec. III-B): rest positions, zero velocities, tool at its
// start, fresh observed vertices (Floyd's sampling without replacement from
// the top face, sorted) and target vertex from the env's counter-based streams.
// Episode reset of one env by its CTA (Sec. III-B): rest positions, zero
// velocities, tool at its start, fresh observed vertices (Floyd's sampling
// without replacement from the top face, sorted) and target vertex from the
// counter-based streams of `seed`.
__device__ void reset_env(const SimDev& S, int env, unsigned long long seed) {
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
        const unsigned long long st = env_stream(seed, ed.gid, 1u);
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
        const int tgt = M.top[splitmix64_nth(env_stream(seed, ed.gid, 2u), 0ull) %
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
        S.clamp_angle[env] = S.clamp_angle0;
        S.clamp_cs[env] = S.clamp_cs0;
        S.grasp_v[env] = -1;
        S.grasp_d0[env] = 0.f;
    }
}

__global__ void reset_kernel(SimDev S, const uint8_t* __restrict__ mask, unsigned long long seed) {
    const int env = blockIdx.x;
    if (mask && !mask[env]) return;
    reset_env(S, env, seed);
    if (threadIdx.x == 0) {
        S.seed0[env] = seed;
        S.episode[env] = 0;
        S.done_flag[env] = 0;
    }
}

// Auto-reset: an env whose last step reported done starts episode k + 1 with
// the draws of seed splitmix64_nth(seed0, 2^40 + k + 1).
__global__ void auto_reset_kernel(SimDev S) {
    const int env = blockIdx.x;
    const bool was_done = S.done_flag[env] != 0;
    __syncthreads();   // every thread has read the flag before thread 0 clears it
    if (!was_done) return;
    const int k = S.episode[env] + 1;
    reset_env(S, env, splitmix64_nth(S.seed0[env], (1ull << 40) + (unsigned long long)k));
    if (threadIdx.x == 0) {
        S.episode[env] = k;
        S.done_flag[env] = 0;
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

template <int SUB, int ENVS, bool RES, bool RING, int OCC = 0>
static cudaError_t configure_one(size_t smem) {
    // Raise the kernel's dynamic shared-memory limit to what a launch needs
    // (the limit plus the kernel's static shared memory must stay within the
    // device's per-block opt-in maximum).
    static size_t configured = 48 * 1024;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(xpbd_step_kernel<SUB, ENVS, RES, RING, OCC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    return cudaSuccess;
}

template <int SUB, int ENVS, bool RES, bool RING, int OCC = 0>
static cudaError_t launch_one(const SimDev& S, const int* env_list, int n_list, size_t smem, cudaStream_t st,
                              const float* actions, float* obs, float* reward, uint8_t* done) {
    const cudaError_t ce = configure_one<SUB, ENVS, RES, RING, OCC>(smem);
    if (ce != cudaSuccess) return ce;
    const int n_blocks = (n_list + ENVS - 1) / ENVS;
    xpbd_step_kernel<SUB, ENVS, RES, RING, OCC>
        <<<n_blocks, SUB * ENVS, smem, st>>>(S, env_list, n_list, actions, obs, reward, done);
    return cudaGetLastError();
}

bool step_config_supported(int sub, int envs, bool resident, bool ring, int occ) {
    if (occ) return occ == 4 && sub == 256 && envs == 1 && resident && ring;   // 64 registers, 4 CTAs per SM
    if (envs == 1) return sub == 128 || sub == 256 || sub == 384 || sub == 512 || sub == 1024;
    if (!resident || !ring) return false;
    if (envs == 2) return sub == 128 || sub == 256 || sub == 384 || sub == 512;
    if (envs == 4) return sub == 128 || sub == 256;
    return false;
}

cudaError_t launch_step(const SimDev& S, const StepConfig& c, const int* env_list, int n_list,
                        size_t smem_bytes, cudaStream_t stream, const float* a, float* o, float* r,
                        uint8_t* d) {
    if (n_list <= 0) return cudaSuccess;
    if (c.occ == 4 && c.sub == 256 && c.envs == 1 && c.resident && c.ring)
        return launch_one<256, 1, true, true, 4>(S, env_list, n_list, smem_bytes, stream, a, o, r, d);
    if (c.occ) return cudaErrorInvalidValue;
#define FFSRL_CASE(SUB_, ENVS_, RES_, RING_)                                                      \
    if (c.sub == SUB_ && c.envs == ENVS_ && c.resident == RES_ && c.ring == RING_)                \
        return launch_one<SUB_, ENVS_, RES_, RING_>(S, env_list, n_list, smem_bytes, stream, a, o, r, d);
#define FFSRL_CASE4(SUB_)                                                                         \
    FFSRL_CASE(SUB_, 1, true, true) FFSRL_CASE(SUB_, 1, true, false) FFSRL_CASE(SUB_, 1, false, true) \
    FFSRL_CASE(SUB_, 1, false, false)
    FFSRL_CASE4(128)
    FFSRL_CASE4(256)
    FFSRL_CASE4(384)
    FFSRL_CASE4(512)
    FFSRL_CASE4(1024)
    FFSRL_CASE(128, 2, true, true)
    FFSRL_CASE(256, 2, true, true)
    FFSRL_CASE(384, 2, true, true)
    FFSRL_CASE(512, 2, true, true)
    FFSRL_CASE(128, 4, true, true)
    FFSRL_CASE(256, 4, true, true)
#undef FFSRL_CASE4
#undef FFSRL_CASE
    return cudaErrorInvalidValue;
}

int step_ctas_per_sm(const StepConfig& c) { return c.occ ? c.occ : min_ctas_per_sm(c.sub * c.envs); }

int step_max_active(const StepConfig& c, size_t smem_bytes) {
    int n = 0;
    if (c.occ == 4 && c.sub == 256 && c.envs == 1 && c.resident && c.ring) {
        if (configure_one<256, 1, true, true, 4>(smem_bytes) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, xpbd_step_kernel<256, 1, true, true, 4>, 256,
                                                          smem_bytes) != cudaSuccess)
            return 0;
    }
    return n;
}

cudaError_t configure_step(const StepConfig& c, size_t smem_bytes) {
    if (c.occ == 4 && c.sub == 256 && c.envs == 1 && c.resident && c.ring)
        return configure_one<256, 1, true, true, 4>(smem_bytes);
    if (c.occ) return cudaErrorInvalidValue;
#define FFSRL_CASE(SUB_, ENVS_, RES_, RING_)                                                      \
    if (c.sub == SUB_ && c.envs == ENVS_ && c.resident == RES_ && c.ring == RING_)                \
        return configure_one<SUB_, ENVS_, RES_, RING_>(smem_bytes);
#define FFSRL_CASE4(SUB_)                                                                         \
    FFSRL_CASE(SUB_, 1, true, true) FFSRL_CASE(SUB_, 1, true, false) FFSRL_CASE(SUB_, 1, false, true) \
    FFSRL_CASE(SUB_, 1, false, false)
    FFSRL_CASE4(128)
    FFSRL_CASE4(256)
    FFSRL_CASE4(384)
    FFSRL_CASE4(512)
    FFSRL_CASE4(1024)
    FFSRL_CASE(128, 2, true, true)
    FFSRL_CASE(256, 2, true, true)
    FFSRL_CASE(384, 2, true, true)
    FFSRL_CASE(512, 2, true, true)
    FFSRL_CASE(128, 4, true, true)
    FFSRL_CASE(256, 4, true, true)
#undef FFSRL_CASE4
#undef FFSRL_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_reset(const SimDev& S, const uint8_t* mask, unsigned long long seed, cudaStream_t st) {
    reset_kernel<<<S.n_env, 256, 0, st>>>(S, mask, seed);
    return cudaGetLastError();
}

// New clamp openings: the angle and its cosine and sine, per env.
__global__ void clamp_kernel(SimDev S, const float* angles) {
    const int env = blockIdx.x * blockDim.x + threadIdx.x;
    if (env >= S.n_env) return;
    const float a = angles[env];
    S.clamp_angle[env] = a;
    S.clamp_cs[env] = make_float2(cosf(a), sinf(a));
}

cudaError_t launch_set_clamp(const SimDev& S, const float* angles, cudaStream_t st) {
    clamp_kernel<<<(S.n_env + 255) / 256, 256, 0, st>>>(S, angles);
    return cudaGetLastError();
}

cudaError_t launch_auto_reset(const SimDev& S, cudaStream_t st) {
    auto_reset_kernel<<<S.n_env, 256, 0, st>>>(S);
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
