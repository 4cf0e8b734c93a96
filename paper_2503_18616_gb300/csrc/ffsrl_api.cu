// C ABI of the batched XPBD simulator: creation, reset, step, state access,
// plus the launch planner and autotuner. Contracts are in include/ffsrl.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ffsrl.h"
#include "mesh_setup.h"
#include "mlp_tc.h"
#include "xpbd_device.cuh"
#include "xpbd_launch.h"
#include "xpbd_surrogate.h"

using namespace ffsrl;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

#define FFSRL_CUDA(call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? FFSRL_E_OOM : FFSRL_E_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// One step-kernel launch: the envs of one shared-memory size class (one or
// more meshes, largest envs first) with one execution schedule. Groups run
// concurrently on their own streams.
struct LaunchGroup {
    std::vector<int> meshes;  // distinct meshes of the group
    int n = 0;
    long long verts = 0;      // total vertices (work estimate)
    int* d_list = nullptr;
    std::vector<int> list;    // host copy of the env list
    // mixed rollout (ffsrl_set_surrogate_envs): plain and warm-start sublists
    int* d_plain = nullptr;
    int* d_warm = nullptr;
    int n_plain = 0, n_warm = 0;
    StepConfig cfg;
    bool permute = true;
    int cluster = 0;          // > 1: CTAs per env of the cluster kernel (meshes above one CTA's shared memory)
    bool jacobi = false;      // the Jacobi solver's kernel (FFSRL_SOLVER_JACOBI)
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

// Autotuner choices, cached per mesh size class and batch size for the
// lifetime of the process.
struct TuneKey {
    std::vector<long long> shape;  // (V, E, T, envs) of every mesh of the group
    int substeps, iterations;
    bool operator<(const TuneKey& o) const {
        return std::tie(shape, substeps, iterations) < std::tie(o.shape, o.substeps, o.iterations);
    }
};
struct TuneChoice {
    StepConfig cfg;
    bool permute;
    float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

// Schedules built in this process, keyed by everything build_schedule reads
// (the mesh's positions, masses, tets, connections and tet vertex orders,
// the seed, the variant and the parts): the bank-aware search takes seconds
// on larger meshes, and a process often creates several simulators of one mesh.
std::mutex g_sched_mu;
std::map<std::string, Schedule> g_sched_cache;

template <class T>
void key_append(std::string& k, const std::vector<T>& v) {
    const size_t n = v.size();
    k.append(reinterpret_cast<const char*>(&n), sizeof n);
    k.append(reinterpret_cast<const char*>(v.data()), v.size() * sizeof(T));
}

void cached_schedule(const HostMesh& m, uint64_t seed, bool permute, Schedule& out, int parts = 1) {
    std::string key;
    const long long head[8] = {m.V, m.T, m.E, m.C, (long long)seed, permute, parts, 0};
    key.append(reinterpret_cast<const char*>(head), sizeof head);
    key_append(key, m.rest);
    key_append(key, m.inv_mass);
    key_append(key, m.tet);
    key_append(key, m.conn);
    key_append(key, m.tet_rot);
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        auto it = g_sched_cache.find(key);
        if (it != g_sched_cache.end()) {
            out = it->second;
            return;
        }
    }
    build_schedule(m, seed, permute, out, parts);
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched_cache.emplace(std::move(key), out);
}

const int kSubs[] = {128, 256, 384, 512};
const int kEnvsPerCta[] = {1, 2, 4};

}  // namespace

namespace ffsrl {
// Message of the last failed call on this thread, for the other translation units.
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ffsrl

struct ffsrl_sim {
    int device = 0;
    cudaStream_t stream = nullptr;
    ffsrl_params params{};
    int n_env = 0, obs_dim = 0;
    size_t max_smem = 0;
    std::vector<HostMesh> meshes;
    std::vector<int> env_mesh, voff, pstart;
    std::vector<EnvDev> h_envs;     // per-env descriptors (host copy of S.envs)
    long long stride = 0, total_verts = 0;
    std::vector<void*> dev_allocs;
    float* h_pinned = nullptr;  // staging for ffsrl_step_host
    float* d_stage = nullptr;
    SimDev S{};
    // [0] plain schedule, [1] bank-aware schedule, [2] the bank-aware schedule
    // split for thread-block clusters (meshes of cluster groups; else as [1])
    MeshDev* d_meshes[3] = {nullptr, nullptr, nullptr};
    std::vector<MeshDev> h_meshes[3];
    int* d_pstart = nullptr;
    std::vector<LaunchGroup> groups;
    cudaEvent_t fork = nullptr;
    int resident_envs = 0, ring_envs = 0;
    int n_sm = 0;
    // warm-start network (tensor-core tiles, biases, normalisation)
    bool has_net = false;
    MlpDev net{};
    uint16_t* d_wtiles = nullptr;
    uint16_t* d_btiles = nullptr;
    float* d_bias = nullptr;
    int* d_net_err = nullptr;
    float* d_master = nullptr;    // float32 master parameters
    float* d_adam_m = nullptr;
    float* d_adam_v = nullptr;
    float* d_grad = nullptr;
    float* d_loss = nullptr;
    double* d_norm_acc = nullptr;   // normalisation statistics (38 doubles) and their float32 result (36)
    float* d_norm_out = nullptr;
    int adam_t = 0;
    float norm[FFSRL_NET_NORM] = {};
    // surrogate-assisted substeps (allocated on first use)
    long long lambda_slots = 0;
    float4* d_feat = nullptr;     // [stride][4] features
    float4* d_dx = nullptr;       // [stride] network corrections
    float4* d_vpred = nullptr;    // [stride] predicted velocities (fused warm-start step)
    uint4* d_arows = nullptr;     // network input tiles (fused warm-start step)
    float* d_lambda_full = nullptr;
    // steps with more than one launch replay a captured CUDA graph, one per
    // set of output pointers (a few kept), on a stream of the library's own
    struct StepGraph {
        const float* a;
        float* o;
        float* r;
        uint8_t* d;
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> graphs;
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t graph_in = nullptr, graph_out = nullptr;
    void drop_graphs() {
        for (StepGraph& g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }
    // mixed rollout: warm-start envs stepped beside the plain ones
    bool mixed = false;
    bool has_conn = false;          // some mesh holds tissue connections
    float mix_threshold = 0.f;
    int mix_n_full = 1;
    int* mix_fallbacks = nullptr;
    cudaStream_t warm_stream = nullptr;
    cudaEvent_t warm_done = nullptr;

    template <class T>
    cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) {
            dev_allocs.push_back(q);
            *p = static_cast<T*>(q);
        }
        return e;
    }
    template <class T>
    cudaError_t upload(T** p, const T* src, size_t count) {
        cudaError_t e = alloc(p, count);
        if (e == cudaSuccess && count) e = cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice);
        return e;
    }
    ~ffsrl_sim() {
        for (LaunchGroup& g : groups) {
            if (g.stream) cudaStreamDestroy(g.stream);
            if (g.done) cudaEventDestroy(g.done);
        }
        if (fork) cudaEventDestroy(fork);
        drop_graphs();
        if (graph_stream) cudaStreamDestroy(graph_stream);
        if (graph_in) cudaEventDestroy(graph_in);
        if (graph_out) cudaEventDestroy(graph_out);
        if (warm_stream) cudaStreamDestroy(warm_stream);
        if (warm_done) cudaEventDestroy(warm_done);
        for (void* p : dev_allocs) cudaFree(p);
        if (h_pinned) cudaFreeHost(h_pinned);
    }
};

namespace {

int check_params(const ffsrl_params& p) {
    if (!(p.dt > 0) || !std::isfinite(p.dt)) return fail(FFSRL_E_INVAL, "dt must be > 0");
    if (p.substeps < 1) return fail(FFSRL_E_INVAL, "substeps must be >= 1");
    if (p.iterations < 0) return fail(FFSRL_E_INVAL, "iterations must be >= 0");
    if (!(p.compliance_dist >= 0) || !(p.compliance_vol >= 0))
        return fail(FFSRL_E_INVAL, "compliances must be >= 0");
    if (!(p.tool_radius >= 0)) return fail(FFSRL_E_INVAL, "tool_radius must be >= 0");
    if (p.n_obs_verts < 0) return fail(FFSRL_E_INVAL, "n_obs_verts must be >= 0");
    if (p.max_steps < 0) return fail(FFSRL_E_INVAL, "max_steps must be >= 0");
    const int b = p.block_threads;
    if (b != 0 && b != 128 && b != 256 && b != 384 && b != 512 && b != 1024)
        return fail(FFSRL_E_INVAL, "block_threads must be 0, 128, 256, 384, 512 or 1024");
    if (p.schedule_flags & ~(FFSRL_SCHED_FORCE | FFSRL_SCHED_NO_PERMUTE | FFSRL_SCHED_NO_RING |
                             FFSRL_SCHED_ENVS2 | FFSRL_SCHED_ENVS4 | FFSRL_SCHED_SURROGATE_PIPELINE |
                             FFSRL_SCHED_NO_CLUSTER | FFSRL_SCHED_FOUR_CTAS | FFSRL_SCHED_WARM_STAGED |
                             FFSRL_SCHED_GLOBAL_MEMORY))
        return fail(FFSRL_E_INVAL, "unknown schedule_flags bits");
    if ((p.schedule_flags & FFSRL_SCHED_ENVS2) && (p.schedule_flags & FFSRL_SCHED_ENVS4))
        return fail(FFSRL_E_INVAL, "FFSRL_SCHED_ENVS2 and FFSRL_SCHED_ENVS4 are exclusive");
    if (p.solver != FFSRL_SOLVER_GAUSS_SEIDEL && p.solver != FFSRL_SOLVER_JACOBI)
        return fail(FFSRL_E_INVAL, "solver must be FFSRL_SOLVER_GAUSS_SEIDEL or FFSRL_SOLVER_JACOBI");
    if (p.auto_reset != 0 && p.auto_reset != 1) return fail(FFSRL_E_INVAL, "auto_reset must be 0 or 1");
    if (p.reserved != 0) return fail(FFSRL_E_INVAL, "reserved params must be zero");
    if (p.tool_model != FFSRL_TOOL_SPHERE && p.tool_model != FFSRL_TOOL_GRASPER)
        return fail(FFSRL_E_INVAL, "tool_model must be FFSRL_TOOL_SPHERE or FFSRL_TOOL_GRASPER");
    if (!(p.conn_radius >= 0) || !std::isfinite(p.conn_radius))
        return fail(FFSRL_E_INVAL, "conn_radius must be finite and >= 0");
    if (p.tool_model == FFSRL_TOOL_GRASPER) {
        if (!(p.shaft_radius >= 0) || !(p.clamp_length >= 0) || !(p.clamp_radius >= 0) ||
            !(p.grasp_radius >= 0) || !std::isfinite(p.rcm_height) || !std::isfinite(p.clamp_angle))
            return fail(FFSRL_E_INVAL, "grasper sizes must be finite and >= 0");
        if (p.solver != FFSRL_SOLVER_GAUSS_SEIDEL)
            return fail(FFSRL_E_INVAL, "the grasper runs with the Gauss-Seidel solver");
    }
    return FFSRL_OK;
}

// Upload one mesh's schedule variant and fill its device descriptor.
int upload_mesh(ffsrl_sim* s, const HostMesh& m, const Schedule& sc, MeshDev& d) {
    const ffsrl_params& p = s->params;
    d = MeshDev{};
    d.V = m.V;
    d.Vp = round_up(m.V, 32);
    d.E = m.E;
    d.T = m.T;
    d.n_ecol = sc.n_ephase;   // execution phases (the colours, or their refinement)
    d.n_tcol = sc.n_tphase;
    d.n_top = int(m.top.size());
    d.n_dseg = (sc.n_ephase + sc.n_tphase) * sc.parts;
    d.n_seg = (sc.n_ephase + sc.n_tphase + sc.n_cphase) * sc.parts;
    d.ring_bytes = sc.ring_bytes;
    d.parts = sc.parts;
    d.part_slots = sc.part_slots;
    std::vector<float4> rw(m.V);
    for (int i = 0; i < m.V; ++i)
        rw[i] = make_float4(m.rest[3 * i], m.rest[3 * i + 1], m.rest[3 * i + 2], m.inv_mass[i]);
    unsigned char* d_recs;
    int4* d_segs;
    uint16_t *d_slot, *d_vert;
    float4* d_rw;
    int* d_top;
    FFSRL_CUDA(s->upload(&d_recs, sc.stream.data(), sc.stream.size()));
    FFSRL_CUDA(s->upload(&d_segs, reinterpret_cast<const int4*>(sc.segs.data()), sc.segs.size() / 4));
    FFSRL_CUDA(s->upload(&d_slot, sc.slot_of.data(), sc.slot_of.size()));
    FFSRL_CUDA(s->upload(&d_vert, sc.vert_of.data(), sc.vert_of.size()));
    FFSRL_CUDA(s->upload(&d_rw, rw.data(), rw.size()));
    FFSRL_CUDA(s->upload(&d_top, m.top.data(), m.top.size()));
    d.recs = d_recs;
    d.segs = d_segs;
    if (sc.parts == 1 && d.Vp <= 4096) {
        // the stream again with every slot field x 16 (a byte offset): edge
        // records hold two slots in their first word, tet and connection
        // records in their first two
        std::vector<unsigned char> b16(sc.stream);
        for (int c = 0; c < d.n_seg; ++c) {
            const int32_t* sg = &sc.segs[4 * c];
            const bool edge = c < sc.n_ephase;
            const int rb = edge ? 8 : 16, words = edge ? 1 : 2;
            for (int q = 0; q < sg[2]; ++q)
                for (int w = 0; w < words; ++w) {
                    uint32_t v;
                    unsigned char* at = b16.data() + sg[0] + size_t(q) * rb + 4 * w;
                    std::memcpy(&v, at, 4);
                    v = ((v & 0xFFFFu) << 4) | (((v >> 16) << 4) << 16);
                    std::memcpy(at, &v, 4);
                }
        }
        unsigned char* d_b16;
        FFSRL_CUDA(s->upload(&d_b16, b16.data(), b16.size()));
        d.recs16 = d_b16;
    }
    d.slot_of = d_slot;
    {
        // the warm-start network skips leading 128-slot tiles of pinned vertices
        // (their corrections are never applied)
        int q = 0;
        while (q < m.V && !(m.inv_mass[sc.vert_of[q]] > 0.f)) ++q;
        d.first_free_tile = q / 128;
    }
    d.vert_of = d_vert;
    d.rest_w = d_rw;
    d.top = d_top;
    {
        // 1-ring adjacency (vertices sharing an edge), vertex order
        std::vector<int> off(m.V + 1, 0), nb(2 * size_t(m.E));
        for (int e = 0; e < m.E; ++e) { ++off[m.edge[2 * e] + 1]; ++off[m.edge[2 * e + 1] + 1]; }
        for (int i = 0; i < m.V; ++i) off[i + 1] += off[i];
        std::vector<int> fill(off.begin(), off.end() - 1);
        for (int e = 0; e < m.E; ++e) {
            nb[fill[m.edge[2 * e]]++] = m.edge[2 * e + 1];
            nb[fill[m.edge[2 * e + 1]]++] = m.edge[2 * e];
        }
        int *d_off, *d_nb;
        FFSRL_CUDA(s->upload(&d_off, off.data(), off.size()));
        FFSRL_CUDA(s->upload(&d_nb, nb.data(), nb.size()));
        d.nbr_off = d_off;
        d.nbr = d_nb;
        // the same adjacency indexed by shared-memory slot (fused warm-start
        // step): one 48-byte record per slot, its degree and neighbour slots
        std::vector<float4> rs(m.V);
        int max_deg = 0;
        for (int q = 0; q < m.V; ++q) {
            const int i = sc.vert_of[q];
            max_deg = std::max(max_deg, off[i + 1] - off[i]);
            rs[q] = rw[i];
        }
        std::vector<uint16_t> recs;
        if (max_deg <= kWarmMaxDegree) {
            recs.assign(24 * size_t(m.V), 0);
            for (int q = 0; q < m.V; ++q) {
                const int i = sc.vert_of[q];
                uint16_t* r = &recs[24 * size_t(q)];
                r[0] = uint16_t(off[i + 1] - off[i]);
                for (int k = off[i]; k < off[i + 1]; ++k) r[1 + k - off[i]] = sc.slot_of[nb[k]];
            }
        }
        // how many 128-row network tiles apart a slot and its 1-ring neighbours lie
        int reach = 0;
        for (int q = 0; q < m.V; ++q) {
            const int i = sc.vert_of[q];
            for (int k = off[i]; k < off[i + 1]; ++k)
                reach = std::max(reach, std::abs(q / 128 - int(sc.slot_of[nb[k]]) / 128));
        }
        uint4* d_nr = nullptr;
        float4* d_rs;
        if (!recs.empty())
            FFSRL_CUDA(s->upload(&d_nr, reinterpret_cast<const uint4*>(recs.data()), recs.size() / 8));
        FFSRL_CUDA(s->upload(&d_rs, rs.data(), rs.size()));
        // the records without segment padding (order-free residual sweeps)
        std::vector<uint2> er;
        std::vector<uint4> tr;
        for (int c = 0; c < d.n_dseg; ++c) {   // distance and volume records only
            const int32_t* sg = &sc.segs[4 * c];
            const unsigned char* base = sc.stream.data() + sg[0];
            for (int q = 0; q < sg[2]; ++q) {
                if (c < sc.n_ephase * sc.parts) {
                    uint2 r;
                    std::memcpy(&r, base + 8 * size_t(q), 8);
                    er.push_back(r);
                } else {
                    uint4 r;
                    std::memcpy(&r, base + 16 * size_t(q), 16);
                    tr.push_back(r);
                }
            }
        }
        uint2* d_er;
        uint4* d_tr;
        FFSRL_CUDA(s->upload(&d_er, er.data(), er.size()));
        FFSRL_CUDA(s->upload(&d_tr, tr.data(), tr.size()));
        d.erec = d_er;
        d.trec = d_tr;
        // 1 / (number of constraints containing the vertex), slot order (Jacobi solver)
        std::vector<int> ncons(m.V, 0);
        for (int e = 0; e < m.E; ++e) { ++ncons[m.edge[2 * e]]; ++ncons[m.edge[2 * e + 1]]; }
        for (int t = 0; t < m.T; ++t)
            for (int k = 0; k < 4; ++k) ++ncons[m.tet[4 * t + k]];
        std::vector<float> inv_n(m.V);
        for (int q = 0; q < m.V; ++q) {
            const int n = ncons[sc.vert_of[q]];
            inv_n[q] = n > 0 ? float(1.0 / n) : 0.f;
        }
        float* d_invn;
        FFSRL_CUDA(s->upload(&d_invn, inv_n.data(), inv_n.size()));
        d.inv_ncons = d_invn;
        d.snbr = d_nr;
        d.max_deg = max_deg;
        d.tile_reach = reach;
        d.rest_s = d_rs;
    }
    // Tool box around the rest bounding box and tool start above the top face.
    for (int k = 0; k < 2; ++k) {
        d.box_lo[k] = m.bbmin[k] - p.tool_margin_xy;
        d.box_hi[k] = m.bbmax[k] + p.tool_margin_xy;
        d.tool_start[k] = (m.bbmin[k] + m.bbmax[k]) / 2;
    }
    d.box_lo[2] = m.bbmax[2] - p.tool_margin_below;
    d.box_hi[2] = m.bbmax[2] + p.tool_margin_above;
    // the tool touches the top face: the sphere's lowest point, or the grasper's clamp tips
    d.tool_start[2] = m.bbmax[2] + (p.tool_model == FFSRL_TOOL_GRASPER
                                        ? p.clamp_length * std::cos(p.clamp_angle) + p.clamp_radius
                                        : p.tool_radius);
    d.rcm[0] = float((m.bbmin[0] + m.bbmax[0]) / 2);
    d.rcm[1] = float((m.bbmin[1] + m.bbmax[1]) / 2);
    d.rcm[2] = float(m.bbmax[2] + p.rcm_height);
    {
        // surface faces in colour-major order, as slots (the schedule's records)
        std::vector<uint4> fr(std::max(1, m.F));
        for (int q = 0; q < m.F; ++q)
            fr[q] = make_uint4(sc.frec[4 * size_t(q)], sc.frec[4 * size_t(q) + 1], 0u, 0u);
        uint4* d_fr;
        int* d_fo;
        FFSRL_CUDA(s->upload(&d_fr, fr.data(), fr.size()));
        FFSRL_CUDA(s->upload(&d_fo, m.fcol_off.data(), m.fcol_off.size()));
        d.F = m.F;
        d.n_fcol = m.n_fcol;
        d.frec = d_fr;
        d.fcol_off = d_fo;
    }
    const double min_len = 1e-12 * m.extent;
    d.min_len2 = float(min_len * min_len);
    return FFSRL_OK;
}

// Shared memory a configuration needs, or 0 if it is not compiled or does not fit.
size_t group_smem(const ffsrl_sim* s, const MeshDev& d, const StepConfig& c) {
    if (!step_config_supported(c.sub, c.envs, c.resident, c.ring, c.occ)) return 0;
    const size_t b = step_smem_bytes(d.Vp, c.resident, c.ring, d.ring_bytes, d.n_seg, c.envs);
    if (b + 256 > s->max_smem) return 0;  // room for the kernel's static shared memory
    // the 4-CTA register budget only pays when four CTAs fit an SM's shared
    // memory; that build reads the byte-offset record stream
    if (c.occ && (step_max_active(c, b) < c.occ || !d.recs16)) return 0;
    return b;
}

// Largest shared memory over the meshes of a group (0 if one does not fit).
size_t group_smem(const ffsrl_sim* s, const LaunchGroup& g, bool permute, const StepConfig& c) {
    if (c.envs > 1 && g.meshes.size() > 1) return 0;   // envs of one CTA share one mesh's ring
    size_t mx = 0;
    for (int mi : g.meshes) {
        const size_t b = group_smem(s, s->h_meshes[permute ? 1 : 0][mi], c);
        if (!b) return 0;
        mx = std::max(mx, b);
    }
    return mx;
}

// One group's step kernel over `list` (the group's envs or a sublist).
cudaError_t group_launch(const ffsrl_sim* s, const LaunchGroup& g, SimDev S, const int* list, int n, cudaStream_t st,
                         const float* a, float* o, float* r, uint8_t* d) {
    if (g.cluster > 1) {
        S.meshes = s->d_meshes[2];
        return launch_cluster_step(S, g.cfg.sub, g.cluster, list, n, g.smem, st, a, o, r, d);
    }
    if (g.jacobi) {
        S.meshes = s->d_meshes[1];
        return launch_jacobi_step(S, list, n, g.smem, st, a, o, r, d);
    }
    S.meshes = s->d_meshes[g.permute ? 1 : 0];
    return launch_step(S, g.cfg, list, n, g.smem, st, a, o, r, d);
}

cudaError_t launch_group(ffsrl_sim* s, const LaunchGroup& g, cudaStream_t st, const float* a, float* o, float* r,
                         uint8_t* d) {
    return group_launch(s, g, s->S, g.d_list, g.n, st, a, o, r, d);
}

// All groups of one step: forked onto the groups' streams after the work
// already queued on the sim's stream, joined back before the step returns.
// In a mixed rollout only the plain sublists are launched here.
cudaError_t launch_all(ffsrl_sim* s, const SimDev* Sx, const float* a, float* o, float* r, uint8_t* d,
                       cudaStream_t main) {
    if (s->groups.size() == 1) {
        const LaunchGroup& g = s->groups[0];
        const SimDev S = Sx ? *Sx : s->S;
        return s->mixed ? group_launch(s, g, S, g.d_plain, g.n_plain, main, a, o, r, d)
                        : group_launch(s, g, S, g.d_list, g.n, main, a, o, r, d);
    }
    cudaError_t e = cudaEventRecord(s->fork, main);
    for (const LaunchGroup& g : s->groups) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g.stream, s->fork, 0);
        const SimDev S = Sx ? *Sx : s->S;
        if (e == cudaSuccess)
            e = s->mixed ? group_launch(s, g, S, g.d_plain, g.n_plain, g.stream, a, o, r, d)
                         : group_launch(s, g, S, g.d_list, g.n, g.stream, a, o, r, d);
        if (e == cudaSuccess) e = cudaEventRecord(g.done, g.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, g.done, 0);
    }
    return e;
}

// Times candidate schedules of one group on its own envs (device-drawn
// actions, no outputs) and keeps the fastest: threads per env, envs per CTA,
// the TMA ring and the bank-aware slot permutation. The envs are reset
// afterwards by the caller.
int autotune_group(ffsrl_sim* s, LaunchGroup& g) {
    const ffsrl_params& p = s->params;
    if (g.cluster > 1 || g.jacobi) return FFSRL_OK;   // one compiled schedule
    TuneKey key;
    for (int mi : g.meshes) {
        const HostMesh& m = s->meshes[mi];
        long long cnt = 0;
        for (int e = 0; e < s->n_env; ++e) cnt += s->env_mesh[e] == mi;
        key.shape.insert(key.shape.end(), {m.V, m.E, m.T, cnt});
    }
    key.substeps = p.substeps;
    key.iterations = p.iterations;
    const bool force_sched = (p.schedule_flags & FFSRL_SCHED_FORCE) != 0;
    const bool resident = g.cfg.resident;
    if (!p.block_threads && !force_sched) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && it->second.cfg.resident == resident) {
            g.cfg = it->second.cfg;
            g.permute = it->second.permute;
            g.smem = group_smem(s, g, g.permute, g.cfg);
            if (g.smem) return FFSRL_OK;
        }
    }
    std::vector<StepConfig> cands;
    const bool force_perm = !(p.schedule_flags & FFSRL_SCHED_NO_PERMUTE);
    const bool force_ring = !(p.schedule_flags & FFSRL_SCHED_NO_RING);
    if (force_sched) {
        // one forced candidate: block_threads (default 256) per env, envs per CTA from the flags
        StepConfig c;
        c.sub = p.block_threads ? p.block_threads : 256;
        c.envs = (p.schedule_flags & FFSRL_SCHED_ENVS4) ? 4 : (p.schedule_flags & FFSRL_SCHED_ENVS2) ? 2 : 1;
        c.resident = resident;
        c.ring = force_ring;
        c.occ = (p.schedule_flags & FFSRL_SCHED_FOUR_CTAS) ? 4 : 0;
        cands.push_back(c);
    } else {
        const std::vector<int> subs = p.block_threads ? std::vector<int>{p.block_threads}
                                                      : std::vector<int>(std::begin(kSubs), std::end(kSubs));
        for (int envs : kEnvsPerCta)
            for (int sub : subs)
                for (int ring = 1; ring >= 0; --ring) {
                    StepConfig c;
                    c.sub = sub;
                    c.envs = envs;
                    c.resident = resident;
                    c.ring = ring;
                    cands.push_back(c);
                    if (sub == 256 && envs == 1 && ring && resident) {
                        c.occ = 4;   // the same kernel budgeted for four CTAs per SM
                        cands.push_back(c);
                    }
                }
    }
    std::vector<int> perm_opts = force_sched ? std::vector<int>{force_perm ? 1 : 0} : std::vector<int>{1, 0};
    struct Cand { StepConfig c; bool perm; size_t smem; };
    std::vector<Cand> feasible;
    for (const StepConfig& c : cands)
        for (int pm : perm_opts) {
            const size_t sm = group_smem(s, g, bool(pm), c);
            if (sm) feasible.push_back({c, bool(pm), sm});
        }
    if (feasible.empty()) {
        if (force_sched) return fail(FFSRL_E_INVAL, "the forced step schedule is not available for this mesh");
        return fail(FFSRL_E_INVAL, "no step schedule fits this device");
    }
    TuneChoice best{feasible[0].c, feasible[0].perm, 1e30f};
    if (feasible.size() > 1) {
        cudaEvent_t e0, e1;
        FFSRL_CUDA(cudaEventCreate(&e0));
        FFSRL_CUDA(cudaEventCreate(&e1));
        for (const Cand& cd : feasible) {
            LaunchGroup c = g;
            c.cfg = cd.c;
            c.permute = cd.perm;
            c.smem = cd.smem;
            FFSRL_CUDA(launch_group(s, c, s->stream, nullptr, nullptr, nullptr, nullptr));  // warm-up
            FFSRL_CUDA(cudaEventRecord(e0, s->stream));
            for (int i = 0; i < 2; ++i) FFSRL_CUDA(launch_group(s, c, s->stream, nullptr, nullptr, nullptr, nullptr));
            FFSRL_CUDA(cudaEventRecord(e1, s->stream));
            FFSRL_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            FFSRL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (std::getenv("FFSRL_TUNE_LOG"))
                std::fprintf(stderr, "ffsrl autotune meshes=%zu envs=%d resident=%d: sub=%d envs_per_cta=%d ring=%d occ=%d permute=%d %.3f ms\n",
                             g.meshes.size(), g.n, int(resident), cd.c.sub, cd.c.envs, int(cd.c.ring), cd.c.occ,
                             int(cd.perm), ms / 2);
            if (ms < best.ms) best = {cd.c, cd.perm, ms};
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    g.cfg = best.cfg;
    g.permute = best.permute;
    g.smem = group_smem(s, g, g.permute, g.cfg);
    if (!p.block_threads && !force_sched) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return FFSRL_OK;
}

int build_device(ffsrl_sim* s, const double* env_alpha) {
    const ffsrl_params& p = s->params;
    const int n_env = s->n_env;
    const double h = p.dt / p.substeps;

    int max_optin = 0;
    FFSRL_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
    s->max_smem = size_t(max_optin);
    FFSRL_CUDA(cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device));
    FFSRL_CUDA(s->alloc(&s->d_net_err, 1));
    FFSRL_CUDA(cudaMemset(s->d_net_err, 0, sizeof(int)));

    // Schedules of every mesh in both variants, built on host threads
    // (largest meshes first). The bank-aware variant searches for a while and
    // chooses each tet's vertex order; the mesh keeps those orders, so the
    // plain-order variant, built second, and the cluster variant use them too
    // and every schedule gives the same bits.
    const int n_mesh = int(s->meshes.size());
    std::vector<Schedule> sched(2 * size_t(n_mesh));
    for (int v = 1; v >= 0; --v) {
        std::vector<int> jobs(n_mesh);
        for (int mi = 0; mi < n_mesh; ++mi) jobs[mi] = mi;
        std::stable_sort(jobs.begin(), jobs.end(),
                         [&](int a, int b) { return s->meshes[a].V > s->meshes[b].V; });
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int q; (q = next.fetch_add(1)) < n_mesh;) {
                const HostMesh& m = s->meshes[jobs[q]];
                cached_schedule(m, 0x5EEDull + uint64_t(m.V), v == 1, sched[2 * jobs[q] + v]);
            }
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int n_thr = int(std::min<unsigned>(hw, unsigned(n_mesh)));
        std::vector<std::thread> pool;
        for (int t = 1; t < n_thr; ++t) pool.emplace_back(work);
        work();
        for (std::thread& t : pool) t.join();
        if (v == 1)
            for (int mi = 0; mi < n_mesh; ++mi) s->meshes[mi].tet_rot = sched[2 * mi + 1].tet_rot;
    }
    for (int v = 0; v < 2; ++v) {
        s->h_meshes[v].resize(s->meshes.size());
        for (int mi = 0; mi < n_mesh; ++mi) {
            int rc = upload_mesh(s, s->meshes[mi], sched[2 * mi + v], s->h_meshes[v][mi]);
            if (rc) return rc;
        }
        FFSRL_CUDA(s->upload(&s->d_meshes[v], s->h_meshes[v].data(), s->h_meshes[v].size()));
    }
    const std::vector<MeshDev>& md = s->h_meshes[1];

    // Per-env descriptors and packed/padded offsets.
    std::vector<EnvDev> ev(n_env);
    s->voff.resize(n_env);
    s->pstart.resize(n_env);
    long long voff = 0, pst = 0, loff = 0;
    for (int e = 0; e < n_env; ++e) {
        const MeshDev& d = md[s->env_mesh[e]];
        ev[e].mesh = s->env_mesh[e];
        ev[e].voff = int(voff);
        ev[e].loff = int(loff);
        const double a = env_alpha ? env_alpha[e] : p.compliance_dist;
        ev[e].alpha_d = float(a / (h * h));
        ev[e].gid = (unsigned long long)e;
        s->voff[e] = int(voff);
        s->pstart[e] = int(pst);
        voff += d.Vp;
        pst += d.V;
        loff += d.E + d.T + s->meshes[ev[e].mesh].C;   // multiplier slots (used with more than one iteration)
        if (voff > 0x7fffffffLL || pst > 0x7fffffffLL || loff > 0x7fffffffLL)
            return fail(FFSRL_E_INVAL, "too many vertices in total (more than 2^31 rows)");
    }
    s->stride = voff;
    s->total_verts = pst;
    EnvDev* d_ev;
    FFSRL_CUDA(s->upload(&d_ev, ev.data(), ev.size()));
    s->h_envs = ev;
    FFSRL_CUDA(s->upload(&s->d_pstart, s->pstart.data(), s->pstart.size()));

    SimDev& S = s->S;
    S.meshes = s->d_meshes[1];
    S.envs = d_ev;
    S.n_env = n_env;
    S.obs_dim = s->obs_dim;
    S.stride = s->stride;
    FFSRL_CUDA(s->alloc(&S.x, 3 * size_t(s->stride)));
    FFSRL_CUDA(s->alloc(&S.v, 3 * size_t(s->stride)));
    FFSRL_CUDA(cudaMemset(S.x, 0, 3 * size_t(s->stride) * sizeof(float)));
    FFSRL_CUDA(cudaMemset(S.v, 0, 3 * size_t(s->stride) * sizeof(float)));
    FFSRL_CUDA(s->alloc(&S.pg, 3 * size_t(s->stride)));
    FFSRL_CUDA(s->alloc(&S.tool, 3 * size_t(n_env)));
    FFSRL_CUDA(s->alloc(&S.l_prev, n_env));
    FFSRL_CUDA(s->alloc(&S.t_step, n_env));
    FFSRL_CUDA(s->alloc(&S.seed, n_env));
    FFSRL_CUDA(s->alloc(&S.obs_ids, size_t(n_env) * std::max(1, p.n_obs_verts)));
    FFSRL_CUDA(s->alloc(&S.target, n_env));
    FFSRL_CUDA(s->alloc(&S.n_contacts, n_env));
    FFSRL_CUDA(s->alloc(&S.contacts, size_t(s->stride)));
    FFSRL_CUDA(s->alloc(&S.err, n_env));
    FFSRL_CUDA(cudaMemset(S.err, 0, n_env * sizeof(int)));
    FFSRL_CUDA(s->alloc(&S.done_flag, n_env));
    FFSRL_CUDA(s->alloc(&S.seed0, n_env));
    FFSRL_CUDA(s->alloc(&S.episode, n_env));
    FFSRL_CUDA(cudaMemset(S.done_flag, 0, n_env));
    FFSRL_CUDA(cudaMemset(S.episode, 0, n_env * sizeof(int)));
    S.lambda = nullptr;
    s->lambda_slots = loff;
    if (p.iterations > 1) FFSRL_CUDA(s->alloc(&S.lambda, size_t(loff)));
    S.h = float(h);
    S.inv_h = float(1.0 / h);
    S.gx = float(p.gravity[0]);
    S.gy = float(p.gravity[1]);
    S.gz = float(p.gravity[2]);
    S.alpha_v = float(p.compliance_vol / (h * h));
    S.radius = float(p.tool_radius);
    S.action_scale = p.action_scale;
    S.substeps = p.substeps;
    S.iterations = p.iterations;
    S.n_obs = p.n_obs_verts;
    S.max_steps = p.max_steps;
    S.w_l = p.w_l;
    S.w_d = p.w_d;
    S.w_s = p.w_s;
    S.success_dist = p.success_dist;
    S.tool_model = p.tool_model;
    S.shaft_radius = float(p.shaft_radius);
    S.clamp_length = float(p.clamp_length);
    S.clamp_radius = float(p.clamp_radius);
    S.clamp_angle0 = float(p.clamp_angle);
    S.clamp_cs0 = make_float2(float(std::cos(double(S.clamp_angle0))), float(std::sin(double(S.clamp_angle0))));
    FFSRL_CUDA(s->alloc(&S.clamp_cs, n_env));
    S.grasp_radius = float(p.grasp_radius);
    FFSRL_CUDA(s->alloc(&S.clamp_angle, n_env));
    FFSRL_CUDA(s->alloc(&S.grasp_v, n_env));
    FFSRL_CUDA(s->alloc(&S.grasp_d0, n_env));

    // Launch groups: one per shared-memory size class, i.e. by how many CTAs of
    // a mesh's resident configuration fit on one SM (3 or more, 2, 1, or none:
    // the global-memory variant). Inside a group the largest envs come first.
    int smem_sm = 0;
    FFSRL_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device));
    std::vector<int> mesh_class(md.size());
    for (size_t mi = 0; mi < md.size(); ++mi) {
        StepConfig probe;
        const size_t b = group_smem(s, md[mi], probe);   // 256 threads, resident, ring
        mesh_class[mi] = b ? std::min<int>(3, int(size_t(smem_sm) / (b + 1024))) : 0;
        if (b && mesh_class[mi] == 0) mesh_class[mi] = 1;
        if (p.schedule_flags & FFSRL_SCHED_GLOBAL_MEMORY) mesh_class[mi] = 0;
    }
    // Meshes above one CTA's shared memory: a cluster of 2 or 4 CTAs holds
    // the env on chip (class -CL) when it fits and can be scheduled; else the
    // global-memory variant (class 0).
    std::vector<int> part_slots(md.size(), 0);
    std::vector<size_t> cl_smem(md.size(), 0);
    if (!(p.schedule_flags & (FFSRL_SCHED_NO_CLUSTER | FFSRL_SCHED_GLOBAL_MEMORY)) &&
        p.tool_model == FFSRL_TOOL_SPHERE) {
        for (size_t mi = 0; mi < md.size(); ++mi) {
            if (mesh_class[mi] != 0 || s->meshes[mi].C > 0) continue;
            for (int cl : {2, 4}) {
                const int P = ((md[mi].V + cl - 1) / cl + 31) / 32 * 32;
                const size_t b = cluster_smem_bytes(P);
                if (b + 1024 + 256 > s->max_smem || cluster_max_active(kClusterThreads, cl, b) <= 0) continue;
                mesh_class[mi] = -cl;
                part_slots[mi] = P;
                cl_smem[mi] = b;
                break;
            }
        }
    }
    {
        // schedules split by cluster rank for those meshes
        std::vector<int> todo;
        for (size_t mi = 0; mi < md.size(); ++mi)
            if (mesh_class[mi] < 0) todo.push_back(int(mi));
        std::vector<Schedule> sc(todo.size());
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int q; (q = next.fetch_add(1)) < int(todo.size());) {
                const HostMesh& m = s->meshes[todo[q]];
                cached_schedule(m, 0x5EEDull + uint64_t(m.V), true, sc[q], -mesh_class[todo[q]]);
            }
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < std::min<unsigned>(hw, unsigned(todo.size())); ++t) pool.emplace_back(work);
        work();
        for (std::thread& t : pool) t.join();
        s->h_meshes[2] = s->h_meshes[1];
        for (size_t q = 0; q < todo.size(); ++q) {
            int rc = upload_mesh(s, s->meshes[todo[q]], sc[q], s->h_meshes[2][todo[q]]);
            if (rc) return rc;
        }
        FFSRL_CUDA(s->upload(&s->d_meshes[2], s->h_meshes[2].data(), s->h_meshes[2].size()));
    }
    bool any_streaming = false;
    if (p.solver == FFSRL_SOLVER_JACOBI) {
        // one group of every env: the Jacobi kernel keeps each env in one CTA
        LaunchGroup g;
        g.jacobi = true;
        g.cfg.sub = 256;
        g.cfg.ring = false;
        std::vector<int> list;
        for (int e = 0; e < n_env; ++e) {
            list.push_back(e);
            const int mi = s->env_mesh[e];
            g.verts += md[mi].V;
            if (std::find(g.meshes.begin(), g.meshes.end(), mi) == g.meshes.end()) g.meshes.push_back(mi);
        }
        for (int mi : g.meshes) g.smem = std::max(g.smem, jacobi_smem_bytes(md[mi].Vp));
        if (g.smem + 1024 + 256 > s->max_smem)
            return fail(FFSRL_E_INVAL, "the Jacobi solver needs every env in one CTA's shared memory");
        g.n = n_env;
        FFSRL_CUDA(s->upload(&g.d_list, list.data(), list.size()));
        g.list = list;
        s->groups.push_back(g);
    }
    for (int cls : {3, 2, 1, -2, -4, 0}) {
        if (p.solver == FFSRL_SOLVER_JACOBI) break;
        LaunchGroup g;
        std::vector<std::pair<int, int>> members;   // (-V, env)
        for (int e = 0; e < n_env; ++e)
            if (mesh_class[s->env_mesh[e]] == cls) members.push_back({-md[s->env_mesh[e]].V, e});
        if (members.empty()) continue;
        std::sort(members.begin(), members.end());
        std::vector<int> list;
        for (auto& pr : members) {
            list.push_back(pr.second);
            g.verts += -pr.first;
            const int mi = s->env_mesh[pr.second];
            if (std::find(g.meshes.begin(), g.meshes.end(), mi) == g.meshes.end()) g.meshes.push_back(mi);
        }
        g.n = int(list.size());
        g.cfg.resident = cls != 0;
        any_streaming |= cls == 0;
        if (cls < 0) {
            g.cluster = -cls;
            g.cfg.sub = kClusterThreads;
            g.cfg.ring = false;
            g.permute = true;
            for (int mi : g.meshes) g.smem = std::max(g.smem, cl_smem[mi]);
        }
        FFSRL_CUDA(s->upload(&g.d_list, list.data(), list.size()));
        g.list = list;
        s->groups.push_back(g);
    }
    S.xg = nullptr;
    if (any_streaming) FFSRL_CUDA(s->alloc(&S.xg, size_t(s->stride)));

    // Pinned host staging and device staging for ffsrl_step_host.
    const size_t stage = size_t(n_env) * (3 + s->obs_dim + 1) + (size_t(n_env) + 3) / 4;
    FFSRL_CUDA(cudaMallocHost(&s->h_pinned, stage * sizeof(float)));
    FFSRL_CUDA(s->alloc(&s->d_stage, stage));

    // Every env needs a valid state (tool, target, step count) before the
    // autotuner runs steps on it.
    FFSRL_CUDA(launch_reset(S, nullptr, 0ull, s->stream));
    FFSRL_CUDA(cudaStreamSynchronize(s->stream));
    // Execution schedule per group (autotuned unless forced), largest groups
    // first; each group gets its own stream when there are several.
    std::sort(s->groups.begin(), s->groups.end(),
              [](const LaunchGroup& a, const LaunchGroup& b) { return a.verts > b.verts; });
    if (s->groups.size() > 1) {
        FFSRL_CUDA(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
        for (LaunchGroup& g : s->groups) {
            FFSRL_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
            FFSRL_CUDA(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        }
    }
    for (LaunchGroup& g : s->groups) {
        int rc = autotune_group(s, g);
        if (rc) return rc;
        if (g.cfg.resident) s->resident_envs += g.n;
        if (g.cfg.ring) s->ring_envs += g.n;
    }
    return FFSRL_OK;
}

}  // namespace

extern "C" {

const char* ffsrl_last_error(void) { return g_last_error.c_str(); }

int ffsrl_create(const ffsrl_mesh* meshes, int32_t n_meshes, const int32_t* env_mesh,
                 const double* env_compliance_dist, int32_t n_env, const ffsrl_params* params,
                 void* cuda_stream, ffsrl_sim** out) {
    if (!out) return fail(FFSRL_E_INVAL, "out must be non-NULL");
    *out = nullptr;
    if (!meshes || n_meshes < 1 || n_env < 1 || !params)
        return fail(FFSRL_E_INVAL, "need meshes, n_meshes >= 1, n_env >= 1 and params");
    int rc = check_params(*params);
    if (rc) return rc;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || n_dev < 1)
        return fail(FFSRL_E_CUDA, "no CUDA device available");
    ffsrl_sim* s = new ffsrl_sim();
    s->params = *params;
    s->n_env = n_env;
    s->obs_dim = 3 + 3 * params->n_obs_verts;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&s->device);
    s->meshes.resize(n_meshes);
    for (int i = 0; i < n_meshes; ++i) {
        std::string err;
        rc = build_host_mesh(meshes[i].n_verts, meshes[i].n_tets, meshes[i].rest_pos, meshes[i].inv_mass,
                             meshes[i].tets, s->meshes[i], err, params->conn_radius);
        if (rc) {
            delete s;
            return fail(rc, "mesh " + std::to_string(i) + ": " + err);
        }
        s->has_conn |= s->meshes[i].C > 0;
    }
    if (s->has_conn && params->solver != FFSRL_SOLVER_GAUSS_SEIDEL) {
        delete s;
        return fail(FFSRL_E_INVAL, "tissue connections run with the Gauss-Seidel solver");
    }
    s->env_mesh.assign(n_env, 0);
    for (int e = 0; e < n_env; ++e) {
        if (env_mesh) s->env_mesh[e] = env_mesh[e];
        if (s->env_mesh[e] < 0 || s->env_mesh[e] >= n_meshes) {
            delete s;
            return fail(FFSRL_E_INVAL, "env_mesh entry out of range");
        }
        if (env_compliance_dist && !(env_compliance_dist[e] >= 0)) {
            delete s;
            return fail(FFSRL_E_INVAL, "env compliance must be >= 0");
        }
        if (int(s->meshes[s->env_mesh[e]].top.size()) < params->n_obs_verts) {
            delete s;
            return fail(FFSRL_E_INVAL, "n_obs_verts exceeds the top-face vertex count of a mesh");
        }
    }
    rc = build_device(s, env_compliance_dist);
    if (rc == FFSRL_OK) {
        // Reset after autotuning, which advanced the envs it timed.
        cudaError_t e = launch_reset(s->S, nullptr, 0ull, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->S.err, 0, n_env * sizeof(int), s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = fail(FFSRL_E_CUDA, std::string("initial reset: ") + cudaGetErrorString(e));
    }
    if (rc) {
        delete s;
        return rc;
    }
    *out = s;
    return FFSRL_OK;
}

int ffsrl_destroy(ffsrl_sim* sim) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    cudaSetDevice(sim->device);
    cudaStreamSynchronize(sim->stream);
    delete sim;
    return FFSRL_OK;
}

int ffsrl_reset(ffsrl_sim* sim, const uint8_t* env_mask_dev, uint64_t seed) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(launch_reset(sim->S, env_mask_dev, (unsigned long long)seed, sim->stream));
    return FFSRL_OK;
}

namespace {
int launch_warm_groups(ffsrl_sim* sim, cudaStream_t st, bool sublists, const float* actions, float* obs,
                       float* reward, uint8_t* done, float threshold, int n_full, int* fallbacks, float* residual);
size_t warm_smem(const ffsrl_sim* s, const LaunchGroup& g, bool* jit = nullptr);
}  // namespace

namespace {

// Every launch of one step on `main` (forked onto the group and warm-start
// streams and joined back).
int step_body(ffsrl_sim* sim, cudaStream_t main, const float* a, float* o, float* r, uint8_t* d) {
    if (sim->params.auto_reset) FFSRL_CUDA(launch_auto_reset(sim->S, main));
    if (sim->mixed) {
        // warm-start envs on their own stream, beside the plain groups
        FFSRL_CUDA(cudaEventRecord(sim->fork, main));
        FFSRL_CUDA(cudaStreamWaitEvent(sim->warm_stream, sim->fork, 0));
        const int rc = launch_warm_groups(sim, sim->warm_stream, true, a, o, r, d, sim->mix_threshold,
                                          sim->mix_n_full, sim->mix_fallbacks, nullptr);
        if (rc) return rc;
        FFSRL_CUDA(cudaEventRecord(sim->warm_done, sim->warm_stream));
    }
    FFSRL_CUDA(launch_all(sim, nullptr, a, o, r, d, main));
    if (sim->mixed) FFSRL_CUDA(cudaStreamWaitEvent(main, sim->warm_done, 0));
    return FFSRL_OK;
}

}  // namespace

int ffsrl_step(ffsrl_sim* sim, const float* actions_dev, float* obs_dev, float* reward_dev,
               uint8_t* done_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    if (sim->groups.size() == 1 && !sim->mixed && !sim->params.auto_reset)
        return step_body(sim, sim->stream, actions_dev, obs_dev, reward_dev, done_dev);
    // Several launches: replay the step's CUDA graph for these pointers,
    // capturing it on first use (on the library's stream, so the caller's
    // stream may be the legacy default stream).
    if (!sim->graph_stream) {
        FFSRL_CUDA(cudaStreamCreateWithFlags(&sim->graph_stream, cudaStreamNonBlocking));
        FFSRL_CUDA(cudaEventCreateWithFlags(&sim->graph_in, cudaEventDisableTiming));
        FFSRL_CUDA(cudaEventCreateWithFlags(&sim->graph_out, cudaEventDisableTiming));
    }
    cudaGraphExec_t exec = nullptr;
    for (const ffsrl_sim::StepGraph& g : sim->graphs)
        if (g.a == actions_dev && g.o == obs_dev && g.r == reward_dev && g.d == done_dev) exec = g.exec;
    if (!exec) {
        // kernel attributes are set outside the capture
        for (const LaunchGroup& g : sim->groups) {
            if (g.jacobi) FFSRL_CUDA(configure_jacobi_step(g.smem));
            else if (g.cluster <= 1) FFSRL_CUDA(configure_step(g.cfg, g.smem));
            if (sim->mixed && g.n_warm) {
                bool jit = false;
                const size_t ws = warm_smem(sim, g, &jit);
                FFSRL_CUDA(configure_warm_step(ws, jit));
            }
        }
        FFSRL_CUDA(cudaStreamBeginCapture(sim->graph_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = step_body(sim, sim->graph_stream, actions_dev, obs_dev, reward_dev, done_dev);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(sim->graph_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        FFSRL_CUDA(ec);
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        FFSRL_CUDA(ei);
        if (sim->graphs.size() >= 4) {
            cudaGraphExecDestroy(sim->graphs.front().exec);
            sim->graphs.erase(sim->graphs.begin());
        }
        sim->graphs.push_back({actions_dev, obs_dev, reward_dev, done_dev, exec});
    }
    FFSRL_CUDA(cudaEventRecord(sim->graph_in, sim->stream));
    FFSRL_CUDA(cudaStreamWaitEvent(sim->graph_stream, sim->graph_in, 0));
    FFSRL_CUDA(cudaGraphLaunch(exec, sim->graph_stream));
    FFSRL_CUDA(cudaEventRecord(sim->graph_out, sim->graph_stream));
    FFSRL_CUDA(cudaStreamWaitEvent(sim->stream, sim->graph_out, 0));
    return FFSRL_OK;
}

// Whether p is page-locked host memory (cudaHostAlloc or registered), which
// the copy engines read and write directly.
static bool page_locked(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int ffsrl_step_host(ffsrl_sim* sim, const float* actions_host, float* obs_host, float* reward_host,
                    uint8_t* done_host) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    const size_t n = size_t(sim->n_env), od = size_t(sim->obs_dim);
    float* h_act = sim->h_pinned;
    float* h_obs = h_act + 3 * n;
    float* h_rew = h_obs + od * n;
    uint8_t* h_done = reinterpret_cast<uint8_t*>(h_rew + n);
    float* d_act = sim->d_stage;
    float* d_obs = d_act + 3 * n;
    float* d_rew = d_obs + od * n;
    uint8_t* d_done = reinterpret_cast<uint8_t*>(d_rew + n);
    // Page-locked caller buffers are copied directly; others go through the
    // sim's page-locked staging buffers.
    const bool pa = page_locked(actions_host), po = page_locked(obs_host), pr = page_locked(reward_host),
               pd = page_locked(done_host);
    if (actions_host) {
        if (!pa) std::memcpy(h_act, actions_host, 3 * n * sizeof(float));
        FFSRL_CUDA(cudaMemcpyAsync(d_act, pa ? actions_host : h_act, 3 * n * sizeof(float), cudaMemcpyHostToDevice,
                                   sim->stream));
    }
    int rc = ffsrl_step(sim, actions_host ? d_act : nullptr, obs_host ? d_obs : nullptr,
                        reward_host ? d_rew : nullptr, done_host ? d_done : nullptr);
    if (rc) return rc;
    if (obs_host)
        FFSRL_CUDA(cudaMemcpyAsync(po ? obs_host : h_obs, d_obs, od * n * sizeof(float), cudaMemcpyDeviceToHost,
                                   sim->stream));
    if (reward_host)
        FFSRL_CUDA(cudaMemcpyAsync(pr ? reward_host : h_rew, d_rew, n * sizeof(float), cudaMemcpyDeviceToHost,
                                   sim->stream));
    if (done_host)
        FFSRL_CUDA(cudaMemcpyAsync(pd ? done_host : h_done, d_done, n, cudaMemcpyDeviceToHost, sim->stream));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    if (obs_host && !po) std::memcpy(obs_host, h_obs, od * n * sizeof(float));
    if (reward_host && !pr) std::memcpy(reward_host, h_rew, n * sizeof(float));
    if (done_host && !pd) std::memcpy(done_host, h_done, n);
    return FFSRL_OK;
}

int ffsrl_sync(ffsrl_sim* sim) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    int net_err = 0;
    FFSRL_CUDA(cudaMemcpy(&net_err, sim->d_net_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (net_err) {
        FFSRL_CUDA(cudaMemset(sim->d_net_err, 0, sizeof(int)));
        return fail(FFSRL_E_TIMEOUT, "a tensor-core completion wait of the warm-start network timed out");
    }
    std::vector<int> err(sim->n_env);
    FFSRL_CUDA(cudaMemcpy(err.data(), sim->S.err, err.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int first = -1, bits = 0;
    for (int e = 0; e < sim->n_env; ++e)
        if (err[e]) {
            bits |= err[e];
            if (first < 0) first = e;
        }
    if (first >= 0) {
        FFSRL_CUDA(cudaMemset(sim->S.err, 0, err.size() * sizeof(int)));
        if (bits & kErrTimeout)
            return fail(FFSRL_E_TIMEOUT,
                        "a bounded wait (constraint-record copy or tensor-core completion) timed out in env " +
                            std::to_string(first));
        return fail(FFSRL_E_NAN, "non-finite positions in env " + std::to_string(first));
    }
    return FFSRL_OK;
}

int ffsrl_set_network(ffsrl_sim* sim, const float* params_host, const float* norm_host) {
    if (!sim || !params_host || !norm_host) return fail(FFSRL_E_INVAL, "sim, params and norm must be non-NULL");
    for (int i = 0; i < FFSRL_NET_PARAMS; ++i)
        if (!std::isfinite(params_host[i])) return fail(FFSRL_E_INVAL, "non-finite network parameter");
    for (int i = 0; i < FFSRL_NET_NORM; ++i)
        if (!std::isfinite(norm_host[i])) return fail(FFSRL_E_INVAL, "non-finite normalisation value");
    for (int k = 0; k < 15; ++k)
        if (!(norm_host[15 + k] > 0)) return fail(FFSRL_E_INVAL, "feature std must be > 0");
    for (int k = 0; k < 3; ++k)
        if (!(norm_host[33 + k] > 0)) return fail(FFSRL_E_INVAL, "output std must be > 0");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    if (!sim->d_master) {
        FFSRL_CUDA(sim->alloc(&sim->d_master, FFSRL_NET_PARAMS));
        FFSRL_CUDA(sim->alloc(&sim->d_adam_m, FFSRL_NET_PARAMS));
        FFSRL_CUDA(sim->alloc(&sim->d_adam_v, FFSRL_NET_PARAMS));
        FFSRL_CUDA(sim->alloc(&sim->d_grad, FFSRL_NET_PARAMS));
        FFSRL_CUDA(sim->alloc(&sim->d_loss, 1));
        FFSRL_CUDA(sim->alloc(&sim->d_wtiles, kMlpWeightBytes / 2));
        FFSRL_CUDA(sim->alloc(&sim->d_btiles, 10240 / 2));
        FFSRL_CUDA(sim->alloc(&sim->d_bias, 144));
    }
    FFSRL_CUDA(cudaMemcpyAsync(sim->d_master, params_host, FFSRL_NET_PARAMS * sizeof(float), cudaMemcpyHostToDevice,
                               sim->stream));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_adam_m, 0, FFSRL_NET_PARAMS * sizeof(float), sim->stream));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_adam_v, 0, FFSRL_NET_PARAMS * sizeof(float), sim->stream));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_grad, 0, FFSRL_NET_PARAMS * sizeof(float), sim->stream));
    FFSRL_CUDA(launch_mlp_pack(sim->d_master, sim->d_wtiles, sim->d_btiles, sim->d_bias, sim->stream));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    sim->adam_t = 0;
    std::memcpy(sim->norm, norm_host, sizeof(sim->norm));
    MlpDev& n = sim->net;
    n.wtiles = sim->d_wtiles;
    n.bias = sim->d_bias;
    for (int k = 0; k < 16; ++k) {
        n.in_mean[k] = k < 15 ? norm_host[k] : 0.f;
        n.in_inv_std[k] = k < 15 ? 1.0f / norm_host[15 + k] : 0.f;
    }
    for (int k = 0; k < 4; ++k) {
        n.out_mean[k] = k < 3 ? norm_host[30 + k] : 0.f;
        n.out_std[k] = k < 3 ? norm_host[33 + k] : 0.f;
    }
    sim->has_net = true;
    sim->drop_graphs();   // captured steps hold the previous network's normalisation
    return FFSRL_OK;
}

int ffsrl_get_network(const ffsrl_sim* sim, float* params_host) {
    if (!sim || !params_host) return fail(FFSRL_E_INVAL, "sim and params must be non-NULL");
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    FFSRL_CUDA(cudaMemcpy(params_host, sim->d_master, FFSRL_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return FFSRL_OK;
}

namespace {

int check_batch(const ffsrl_sim* sim, const float* f, const float* t, const float* w, int64_t rows, float wsum) {
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    if (rows < 1 || !f || !t || !w) return fail(FFSRL_E_INVAL, "need rows >= 1 and features, targets, weights");
    if (!(wsum > 0)) return fail(FFSRL_E_INVAL, "weight_sum must be > 0");
    if ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(t)) & 15)
        return fail(FFSRL_E_INVAL, "features and targets must be 16-byte aligned");
    return FFSRL_OK;
}

TrainDev train_dev(ffsrl_sim* sim, float wsum) {
    TrainDev P{};
    P.wtiles = sim->d_wtiles;
    P.btiles = sim->d_btiles;
    P.bias = sim->d_bias;
    for (int k = 0; k < 16; ++k) {
        P.in_mean[k] = sim->net.in_mean[k];
        P.in_inv_std[k] = sim->net.in_inv_std[k];
    }
    for (int k = 0; k < 4; ++k) {
        P.out_mean[k] = k < 3 ? sim->norm[30 + k] : 0.f;
        P.out_inv_std[k] = k < 3 ? 1.0f / sim->norm[33 + k] : 0.f;
    }
    P.grad_scale = 2.0f / (3.0f * wsum);
    P.grad = sim->d_grad;
    P.loss = sim->d_loss;
    return P;
}

}  // namespace

int ffsrl_network_gradient(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                           const float* row_weight_dev, int64_t rows, float weight_sum, float* grad_dev,
                           float* loss_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    int rc = check_batch(sim, features_dev, targets_dev, row_weight_dev, rows, weight_sum);
    if (rc) return rc;
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_grad, 0, FFSRL_NET_PARAMS * sizeof(float), sim->stream));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_loss, 0, sizeof(float), sim->stream));
    FFSRL_CUDA(launch_mlp_train(train_dev(sim, weight_sum), reinterpret_cast<const float4*>(features_dev),
                                reinterpret_cast<const float4*>(targets_dev), row_weight_dev, rows, sim->d_net_err,
                                sim->n_sm, sim->stream));
    if (grad_dev)
        FFSRL_CUDA(cudaMemcpyAsync(grad_dev, sim->d_grad, FFSRL_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice,
                                   sim->stream));
    if (loss_dev) FFSRL_CUDA(cudaMemcpyAsync(loss_dev, sim->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, sim->stream));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_grad, 0, FFSRL_NET_PARAMS * sizeof(float), sim->stream));
    return FFSRL_OK;
}

int ffsrl_train_network(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                        const float* row_weight_dev, int64_t rows, float weight_sum, float lr, float* loss_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    int rc = check_batch(sim, features_dev, targets_dev, row_weight_dev, rows, weight_sum);
    if (rc) return rc;
    if (!(lr > 0)) return fail(FFSRL_E_INVAL, "lr must be > 0");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaMemsetAsync(sim->d_loss, 0, sizeof(float), sim->stream));
    FFSRL_CUDA(launch_mlp_train(train_dev(sim, weight_sum), reinterpret_cast<const float4*>(features_dev),
                                reinterpret_cast<const float4*>(targets_dev), row_weight_dev, rows, sim->d_net_err,
                                sim->n_sm, sim->stream));
    sim->adam_t += 1;
    FFSRL_CUDA(launch_adam(sim->d_master, sim->d_adam_m, sim->d_adam_v, sim->d_grad, FFSRL_NET_PARAMS, lr,
                           sim->adam_t, sim->stream));
    FFSRL_CUDA(launch_mlp_pack(sim->d_master, sim->d_wtiles, sim->d_btiles, sim->d_bias, sim->stream));
    if (loss_dev) FFSRL_CUDA(cudaMemcpyAsync(loss_dev, sim->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, sim->stream));
    return FFSRL_OK;
}

int ffsrl_network_adam_step(ffsrl_sim* sim, const float* grad_dev, float lr) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    if (!grad_dev) return fail(FFSRL_E_INVAL, "grad_dev must be non-NULL");
    if (!(lr > 0)) return fail(FFSRL_E_INVAL, "lr must be > 0");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaMemcpyAsync(sim->d_grad, grad_dev, FFSRL_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice,
                               sim->stream));
    sim->adam_t += 1;
    FFSRL_CUDA(launch_adam(sim->d_master, sim->d_adam_m, sim->d_adam_v, sim->d_grad, FFSRL_NET_PARAMS, lr,
                           sim->adam_t, sim->stream));
    FFSRL_CUDA(launch_mlp_pack(sim->d_master, sim->d_wtiles, sim->d_btiles, sim->d_bias, sim->stream));
    return FFSRL_OK;
}

int ffsrl_network_normalisation(ffsrl_sim* sim, const float* features_dev, const float* targets_dev,
                                const float* row_weight_dev, int64_t rows, float* norm_host) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (rows < 1 || !features_dev || !targets_dev || !row_weight_dev || !norm_host)
        return fail(FFSRL_E_INVAL, "need rows >= 1 and features, targets, weights and norm_host");
    if ((reinterpret_cast<uintptr_t>(features_dev) | reinterpret_cast<uintptr_t>(targets_dev)) & 15)
        return fail(FFSRL_E_INVAL, "features and targets must be 16-byte aligned");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    if (!sim->d_norm_acc) {
        FFSRL_CUDA(sim->alloc(&sim->d_norm_acc, 38));
        FFSRL_CUDA(sim->alloc(&sim->d_norm_out, FFSRL_NET_NORM));
    }
    FFSRL_CUDA(launch_norm_stats(reinterpret_cast<const float4*>(features_dev),
                                 reinterpret_cast<const float4*>(targets_dev), row_weight_dev, rows, sim->d_norm_acc,
                                 sim->d_norm_out, sim->n_sm, sim->stream));
    double count = 0;
    FFSRL_CUDA(cudaMemcpyAsync(&count, sim->d_norm_acc + 18, sizeof(double), cudaMemcpyDeviceToHost, sim->stream));
    FFSRL_CUDA(cudaMemcpyAsync(norm_host, sim->d_norm_out, FFSRL_NET_NORM * sizeof(float), cudaMemcpyDeviceToHost,
                               sim->stream));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    if (!(count > 0)) return fail(FFSRL_E_INVAL, "no row has a positive weight");
    for (int i = 0; i < FFSRL_NET_NORM; ++i)
        if (!std::isfinite(norm_host[i])) return fail(FFSRL_E_NAN, "non-finite feature or target in the batch");
    return FFSRL_OK;
}

int ffsrl_network_forward(ffsrl_sim* sim, const float* features_dev, float* out_dev, int64_t rows) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    if (rows < 0 || (rows > 0 && (!features_dev || !out_dev))) return fail(FFSRL_E_INVAL, "bad rows or buffers");
    if ((reinterpret_cast<uintptr_t>(features_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 15)
        return fail(FFSRL_E_INVAL, "features and output must be 16-byte aligned");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(launch_mlp_forward(sim->net, reinterpret_cast<const float4*>(features_dev),
                                  reinterpret_cast<float4*>(out_dev), rows, sim->d_net_err, sim->n_sm, sim->stream));
    return FFSRL_OK;
}

namespace {

int ensure_surrogate_buffers(ffsrl_sim* sim) {
    if (sim->d_feat) return FFSRL_OK;
    FFSRL_CUDA(sim->alloc(&sim->d_feat, 4 * size_t(sim->stride)));
    FFSRL_CUDA(sim->alloc(&sim->d_dx, size_t(sim->stride)));
    FFSRL_CUDA(sim->alloc(&sim->d_vpred, size_t(sim->stride)));
    FFSRL_CUDA(sim->alloc(&sim->d_arows, 2 * (size_t(sim->stride) + 128 * size_t(sim->n_env))));
    FFSRL_CUDA(cudaMemset(sim->d_feat, 0, 4 * size_t(sim->stride) * sizeof(float4)));
    FFSRL_CUDA(cudaMemset(sim->d_dx, 0, size_t(sim->stride) * sizeof(float4)));
    FFSRL_CUDA(sim->alloc(&sim->d_lambda_full, size_t(sim->lambda_slots)));
    if (!sim->S.xg) {
        // the per-substep pipeline runs cluster groups on the global working copy
        bool need = false;
        for (const LaunchGroup& g : sim->groups) need |= !g.cfg.resident || g.cluster > 1;
        if (need) FFSRL_CUDA(sim->alloc(&sim->S.xg, size_t(sim->stride)));
    }
    return FFSRL_OK;
}

// Shared memory of the substep kernel for a group (0: not resident).
size_t substep_smem(const ffsrl_sim* s, const LaunchGroup& g, bool& resident) {
    int vp = 0;
    for (int mi : g.meshes) vp = std::max(vp, s->h_meshes[1][mi].Vp);
    const size_t res = substep_smem_bytes(vp, true);
    resident = g.cfg.resident && res + 256 <= s->max_smem;
    return resident ? res : substep_smem_bytes(vp, false);
}

// Shared memory of the fused warm-start step for a group (0: does not fit),
// and in *jit which of its two kernels runs: the just-in-time one where every
// mesh's 1-ring spans at most kWarmJitMaxReach tiles and it fits (unless
// FFSRL_SCHED_WARM_STAGED), else the staged one.
size_t warm_smem(const ffsrl_sim* s, const LaunchGroup& g, bool* jit) {
    size_t b_jit = 0, b_st = 0;
    bool can_jit = !(s->params.schedule_flags & FFSRL_SCHED_WARM_STAGED);
    for (int mi : g.meshes) {
        const MeshDev& d = s->h_meshes[g.permute ? 1 : 0][mi];
        if (d.max_deg > kWarmMaxDegree) return 0;
        can_jit &= d.tile_reach <= kWarmJitMaxReach;
        b_jit = std::max(b_jit, warm_smem_bytes(d.Vp, d.ring_bytes, d.n_seg, true));
        b_st = std::max(b_st, warm_smem_bytes(d.Vp, d.ring_bytes, d.n_seg, false));
    }
    const size_t room = 1024 + 256;   // the kernels' static shared memory
    const bool use_jit = can_jit && b_jit + room <= s->max_smem;
    if (jit) *jit = use_jit;
    if (use_jit) return b_jit;
    return b_st + room <= s->max_smem ? b_st : 0;
}

// Residual evaluation and fallback decision of a warm-start substep: a
// threshold of +inf never falls back (and the residual is evaluated only if
// it is requested); any other threshold falls back unless the residual is at
// most the threshold (a NaN residual falls back).
void set_residual_flags(SubstepCtl& C, float threshold, const float* residual) {
    C.decide = !(std::isinf(threshold) && threshold > 0) ? 1 : 0;
    C.check = (C.decide || residual) ? 1 : 0;
}

// Fused warm-start steps of the groups that fit (all envs of each group, or
// their warm-start sublists in a mixed rollout).
int launch_warm_groups(ffsrl_sim* sim, cudaStream_t st, bool sublists, const float* actions, float* obs,
                       float* reward, uint8_t* done, float threshold, int n_full, int* fallbacks, float* residual) {
    SubstepCtl C{};
    C.mode = kSubstepSurrogate;
    C.threshold = threshold;
    set_residual_flags(C, threshold, residual);
    C.n_full = n_full;
    C.lambda = sim->d_lambda_full;
    C.fallbacks = fallbacks;
    C.residual = residual;
    C.scratch = sim->d_dx;
    C.vpred = sim->d_vpred;
    C.arows = sim->d_arows;
    for (const LaunchGroup& g : sim->groups) {
        const int n = sublists ? g.n_warm : g.n;
        bool jit = false;
        const size_t smem = warm_smem(sim, g, &jit);
        if (!n || !smem) continue;
        SimDev S = sim->S;
        S.meshes = sim->d_meshes[g.permute ? 1 : 0];
        FFSRL_CUDA(launch_warm_step(S, sim->net, C, sublists ? g.d_warm : g.d_list, n, smem, jit, actions, obs,
                                    reward, done, st));
    }
    return FFSRL_OK;
}

// One surrogate or record step of every env. Surrogate mode: groups that fit
// the fused kernel take one launch; the others (and every group in record mode
// or with FFSRL_SCHED_SURROGATE_PIPELINE) per substep the features, the network
// and the substep kernel.
int run_substeps(ffsrl_sim* sim, int mode, const float* actions, float* obs, float* reward, uint8_t* done,
                 float threshold, int n_full, int* fallbacks, float* residual, float* feat_out, float* target_out) {
    if (sim->params.solver != FFSRL_SOLVER_GAUSS_SEIDEL || sim->params.tool_model != FFSRL_TOOL_SPHERE ||
        sim->has_conn)
        return fail(FFSRL_E_INVAL,
                    "the warm-start and recording steps use the Gauss-Seidel solve, the sphere tool and no connections");
    int rc = ensure_surrogate_buffers(sim);
    if (rc) return rc;
    if (sim->params.auto_reset) FFSRL_CUDA(launch_auto_reset(sim->S, sim->stream));
    const int S_sub = sim->params.substeps;
    const size_t rows = size_t(sim->stride);
    const bool fused = mode == kSubstepSurrogate && !(sim->params.schedule_flags & FFSRL_SCHED_SURROGATE_PIPELINE);
    std::vector<const LaunchGroup*> pipe;
    for (const LaunchGroup& g : sim->groups)
        if (!fused || !warm_smem(sim, g)) pipe.push_back(&g);
    if (fused) {
        rc = launch_warm_groups(sim, sim->stream, false, actions, obs, reward, done, threshold, n_full, fallbacks,
                                residual);
        if (rc) return rc;
    }
    if (pipe.empty()) return FFSRL_OK;
    for (int sub = 0; sub < S_sub; ++sub) {
        float4* F = feat_out ? reinterpret_cast<float4*>(feat_out) + size_t(sub) * rows * 4 : sim->d_feat;
        for (const LaunchGroup* gp : pipe) {
            const LaunchGroup& g = *gp;
            SimDev S = sim->S;
            S.meshes = sim->d_meshes[g.permute ? 1 : 0];
            FFSRL_CUDA(launch_features(S, g.d_list, g.n, sub == 0, actions, F, sim->stream));
        }
        if (mode == kSubstepSurrogate)
            FFSRL_CUDA(launch_mlp_forward(sim->net, F, sim->d_dx, (long long)rows, sim->d_net_err, sim->n_sm,
                                          sim->stream));
        SubstepCtl C{};
        C.mode = mode;
        C.last = sub == S_sub - 1;
        C.dx = sim->d_dx;
        C.target = target_out ? reinterpret_cast<float4*>(target_out) + size_t(sub) * rows : nullptr;
        C.threshold = threshold;
        set_residual_flags(C, threshold, residual);
        C.n_full = n_full;
        C.lambda = sim->d_lambda_full;
        C.fallbacks = fallbacks;
        C.residual = residual;
        for (const LaunchGroup* gp : pipe) {
            const LaunchGroup& g = *gp;
            SimDev S = sim->S;
            S.meshes = sim->d_meshes[g.permute ? 1 : 0];
            bool resident = false;
            const size_t smem = substep_smem(sim, g, resident);
            FFSRL_CUDA(launch_substep(S, C, g.d_list, g.n, resident, smem, sim->stream, C.last ? obs : nullptr,
                                      C.last ? reward : nullptr, C.last ? done : nullptr));
        }
    }
    return FFSRL_OK;
}

}  // namespace

int ffsrl_step_surrogate(ffsrl_sim* sim, const float* actions_dev, float* obs_dev, float* reward_dev,
                         uint8_t* done_dev, double threshold, int32_t n_full, int32_t* fallbacks_dev,
                         float* residual_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    if (n_full < 1) return fail(FFSRL_E_INVAL, "n_full must be >= 1");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    return run_substeps(sim, kSubstepSurrogate, actions_dev, obs_dev, reward_dev, done_dev, float(threshold), n_full,
                        fallbacks_dev, residual_dev, nullptr, nullptr);
}

int ffsrl_set_surrogate_envs(ffsrl_sim* sim, const uint8_t* mask_host, double threshold, int32_t n_full,
                             int32_t* fallbacks_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    sim->drop_graphs();   // captured steps hold the previous lists and threshold
    if (!mask_host) {
        sim->mixed = false;
        return FFSRL_OK;
    }
    if (!sim->has_net) return fail(FFSRL_E_INVAL, "no network installed (ffsrl_set_network)");
    if (n_full < 1) return fail(FFSRL_E_INVAL, "n_full must be >= 1");
    if (sim->params.solver != FFSRL_SOLVER_GAUSS_SEIDEL || sim->params.tool_model != FFSRL_TOOL_SPHERE ||
        sim->has_conn)
        return fail(FFSRL_E_INVAL, "the warm-start step uses the Gauss-Seidel solve, the sphere tool and no connections");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    int rc = ensure_surrogate_buffers(sim);
    if (rc) return rc;
    for (const LaunchGroup& g : sim->groups) {
        bool any = false;
        for (int e : g.list) any |= mask_host[e] != 0;
        if (any && !warm_smem(sim, g))
            return fail(FFSRL_E_INVAL, "a warm-start env's mesh does not fit the fused kernel's shared memory");
    }
    if (!sim->warm_stream) {
        FFSRL_CUDA(cudaStreamCreateWithFlags(&sim->warm_stream, cudaStreamNonBlocking));
        FFSRL_CUDA(cudaEventCreateWithFlags(&sim->warm_done, cudaEventDisableTiming));
    }
    if (!sim->fork) FFSRL_CUDA(cudaEventCreateWithFlags(&sim->fork, cudaEventDisableTiming));
    for (LaunchGroup& g : sim->groups) {
        std::vector<int> plain, warm;
        for (int e : g.list) (mask_host[e] ? warm : plain).push_back(e);
        if (!g.d_plain) {
            FFSRL_CUDA(sim->alloc(&g.d_plain, g.list.size()));
            FFSRL_CUDA(sim->alloc(&g.d_warm, g.list.size()));
        }
        FFSRL_CUDA(cudaMemcpy(g.d_plain, plain.data(), plain.size() * sizeof(int), cudaMemcpyHostToDevice));
        FFSRL_CUDA(cudaMemcpy(g.d_warm, warm.data(), warm.size() * sizeof(int), cudaMemcpyHostToDevice));
        g.n_plain = int(plain.size());
        g.n_warm = int(warm.size());
    }
    sim->mix_threshold = float(threshold);
    sim->mix_n_full = n_full;
    sim->mix_fallbacks = fallbacks_dev;
    sim->mixed = true;
    return FFSRL_OK;
}

int ffsrl_set_env_ids(ffsrl_sim* sim, const int64_t* ids_host) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    std::vector<EnvDev> ev = sim->h_envs;
    for (int e = 0; e < sim->n_env; ++e) {
        const int64_t id = ids_host ? ids_host[e] : int64_t(e);
        if (id < 0 || id >= (int64_t(1) << 40))
            return fail(FFSRL_E_INVAL, "env ids must lie in [0, 2^40)");
        ev[e].gid = (unsigned long long)id;
    }
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    FFSRL_CUDA(cudaMemcpy(const_cast<EnvDev*>(sim->S.envs), ev.data(), ev.size() * sizeof(EnvDev),
                          cudaMemcpyHostToDevice));
    sim->h_envs = ev;
    return FFSRL_OK;
}

int ffsrl_set_clamp_angles(ffsrl_sim* sim, const float* angles_dev) {
    if (!sim || !angles_dev) return fail(FFSRL_E_INVAL, "sim and angles_dev must be non-NULL");
    if (sim->params.tool_model != FFSRL_TOOL_GRASPER) return fail(FFSRL_E_INVAL, "the sim has no grasper tool");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(launch_set_clamp(sim->S, angles_dev, sim->stream));
    return FFSRL_OK;
}

int ffsrl_get_grasp(ffsrl_sim* sim, int32_t* grasp_host) {
    if (!sim || !grasp_host) return fail(FFSRL_E_INVAL, "sim and grasp_host must be non-NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    FFSRL_CUDA(cudaMemcpy(grasp_host, sim->S.grasp_v, size_t(sim->n_env) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return FFSRL_OK;
}

int ffsrl_record_step(ffsrl_sim* sim, const float* actions_dev, int32_t n_full, float* features_dev,
                      float* targets_dev, float* residual_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (n_full < 1) return fail(FFSRL_E_INVAL, "n_full must be >= 1");
    if ((reinterpret_cast<uintptr_t>(features_dev) | reinterpret_cast<uintptr_t>(targets_dev)) & 15)
        return fail(FFSRL_E_INVAL, "features and targets must be 16-byte aligned");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    return run_substeps(sim, kSubstepRecord, actions_dev, nullptr, nullptr, nullptr, 0.f, n_full, nullptr,
                        residual_dev, features_dev, targets_dev);
}

int ffsrl_get_rows(const ffsrl_sim* sim, int64_t* n_rows, int32_t* row_off_host) {
    if (!sim || !n_rows) return fail(FFSRL_E_INVAL, "sim and n_rows must be non-NULL");
    *n_rows = sim->stride;
    if (row_off_host) std::memcpy(row_off_host, sim->voff.data(), sim->voff.size() * sizeof(int32_t));
    return FFSRL_OK;
}

int ffsrl_get_info(const ffsrl_sim* sim, ffsrl_info* out) {
    if (!sim || !out) return fail(FFSRL_E_INVAL, "sim and out must be non-NULL");
    out->n_env = sim->n_env;
    out->n_meshes = int(sim->meshes.size());
    out->obs_dim = sim->obs_dim;
    int mv = 0;
    for (const HostMesh& m : sim->meshes) mv = std::max(mv, m.V);
    out->max_verts = mv;
    out->total_verts = sim->total_verts;
    out->block_threads = sim->groups.empty() ? 0 : sim->groups.front().cfg.sub;
    out->envs_per_cta = sim->groups.empty() ? 0 : sim->groups.front().cfg.envs;
    out->ctas_per_sm = sim->groups.empty() ? 0 : step_ctas_per_sm(sim->groups.front().cfg);
    out->resident_envs = sim->resident_envs;
    out->n_groups = int(sim->groups.size());
    out->ring_envs = sim->ring_envs;
    return FFSRL_OK;
}

int ffsrl_get_state(ffsrl_sim* sim, float* x_dev, float* v_dev, double* tool_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    if (x_dev || v_dev) FFSRL_CUDA(launch_pack(sim->S, sim->d_pstart, x_dev, v_dev, sim->stream));
    if (tool_dev)
        FFSRL_CUDA(cudaMemcpyAsync(tool_dev, sim->S.tool, 3 * size_t(sim->n_env) * sizeof(double),
                                   cudaMemcpyDeviceToDevice, sim->stream));
    return FFSRL_OK;
}

int ffsrl_set_state(ffsrl_sim* sim, const float* x_dev, const float* v_dev, const double* tool_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    if (x_dev || v_dev) FFSRL_CUDA(launch_unpack(sim->S, sim->d_pstart, x_dev, v_dev, sim->stream));
    if (tool_dev)
        FFSRL_CUDA(cudaMemcpyAsync(sim->S.tool, tool_dev, 3 * size_t(sim->n_env) * sizeof(double),
                                   cudaMemcpyDeviceToDevice, sim->stream));
    return FFSRL_OK;
}

int ffsrl_get_mesh_table(const ffsrl_sim* sim, int32_t mesh, int32_t which, int32_t* out_host,
                         int64_t* count) {
    if (!sim || !count) return fail(FFSRL_E_INVAL, "sim and count must be non-NULL");
    if (mesh < 0 || mesh >= int(sim->meshes.size())) return fail(FFSRL_E_INVAL, "mesh index out of range");
    const HostMesh& m = sim->meshes[mesh];
    const std::vector<int32_t>* src = nullptr;
    switch (which) {
    case 0: src = &m.tet; break;
    case 1: src = &m.flipped; break;
    case 2: src = &m.edge; break;
    case 3: src = &m.ecolor; break;
    case 4: src = &m.tcolor; break;
    case 5: src = &m.eorder; break;
    case 6: src = &m.torder; break;
    case 7: src = &m.ecol_off; break;
    case 8: src = &m.tcol_off; break;
    case 9: src = &m.top; break;
    case 10: src = &m.face; break;
    case 11: src = &m.fopp; break;
    case 12: src = &m.forder; break;
    case 13: src = &m.fcol_off; break;
    case 14: src = &m.conn; break;
    case 15: src = &m.corder; break;
    case 16: src = &m.ccol_off; break;
    case 17: src = &m.obj; break;
    default: return fail(FFSRL_E_INVAL, "unknown table");
    }
    *count = int64_t(src->size());
    if (out_host && !src->empty()) std::memcpy(out_host, src->data(), src->size() * sizeof(int32_t));
    return FFSRL_OK;
}

int ffsrl_get_env_ints(ffsrl_sim* sim, int32_t env, int32_t* step_count, int32_t* target,
                       int32_t* obs_ids_host, int32_t* n_contacts, int32_t* contacts_host) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (env < 0 || env >= sim->n_env) return fail(FFSRL_E_INVAL, "env out of range");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    const SimDev& S = sim->S;
    if (step_count) FFSRL_CUDA(cudaMemcpy(step_count, S.t_step + env, sizeof(int), cudaMemcpyDeviceToHost));
    if (target) FFSRL_CUDA(cudaMemcpy(target, S.target + env, sizeof(int), cudaMemcpyDeviceToHost));
    if (obs_ids_host && sim->params.n_obs_verts > 0)
        FFSRL_CUDA(cudaMemcpy(obs_ids_host, S.obs_ids + size_t(env) * sim->params.n_obs_verts,
                              sim->params.n_obs_verts * sizeof(int), cudaMemcpyDeviceToHost));
    int nc = 0;
    FFSRL_CUDA(cudaMemcpy(&nc, S.n_contacts + env, sizeof(int), cudaMemcpyDeviceToHost));
    if (n_contacts) *n_contacts = nc;
    if (contacts_host && nc > 0)
        FFSRL_CUDA(cudaMemcpy(contacts_host, S.contacts + sim->voff[env], nc * sizeof(int), cudaMemcpyDeviceToHost));
    return FFSRL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free step on caller-owned state (see ffsrl_step_noalloc in
// include/ffsrl.h). Its scratch is this file-scope device array; host code
// reaches it only through the address cudaGetSymbolAddress returns for the
// current device (the symbol itself is a host-side stand-in).
// ---------------------------------------------------------------------------

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FFSRL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current);
// looked up once per device.
int noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return fail(FFSRL_E_CUDA, "device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(FFSRL_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[device];
    return FFSRL_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int ffsrl_step_noalloc(ffsrl_sim* sim, const float* actions_dev, float* x_dev, float* v_dev,
                                  double* tool_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    if (!actions_dev || !x_dev || !v_dev || !tool_dev)
        return fail(FFSRL_E_INVAL, "ffsrl_step_noalloc needs actions_dev, x_dev, v_dev and tool_dev");
    if (sim->mixed) return fail(FFSRL_E_INVAL, "ffsrl_step_noalloc does not step warm-start envs (mixed rollout)");
    if (sim->params.auto_reset) return fail(FFSRL_E_INVAL, "ffsrl_step_noalloc does not auto-reset");
    if (sim->params.tool_model != FFSRL_TOOL_SPHERE)
        return fail(FFSRL_E_INVAL, "ffsrl_step_noalloc steps sims with the sphere tool only (the grasper's grasp "
                                   "state is per-sim state, not caller state)");
    const size_t rows = size_t(sim->stride), n = size_t(sim->n_env);
    bool any_streaming = false;
    for (const LaunchGroup& g : sim->groups) any_streaming |= !g.cfg.resident;
    size_t lam_slots = 0;
    if (sim->params.iterations > 1)
        for (int e = 0; e < sim->n_env; ++e) {
            const HostMesh& m = sim->meshes[sim->env_mesh[e]];
            lam_slots += size_t(m.E + m.T + m.C);
        }
    // Scratch layout: x, v and x_prev ([3][rows] float each), the working
    // positions of non-resident envs ([rows] float4), contacts ([rows] int),
    // per-env counters (step count, contact count, last distance: 3 x [n]
    // int32/float; done flags [n] bytes), multipliers. Error flags are not
    // scratch: they go to the sim's own flags, which ffsrl_sync reports.
    size_t off = 0;
    const size_t o_x = off; off = align256(off + 3 * rows * sizeof(float));
    const size_t o_v = off; off = align256(off + 3 * rows * sizeof(float));
    const size_t o_p = off; off = align256(off + 3 * rows * sizeof(float));
    const size_t o_xg = off; off = align256(off + (any_streaming ? rows * sizeof(float4) : 0));
    const size_t o_c = off; off = align256(off + rows * sizeof(int));
    const size_t o_env = off; off = align256(off + 3 * n * sizeof(int) + n);
    const size_t o_lam = off; off = align256(off + lam_slots * sizeof(float));
    if (off > size_t(FFSRL_NOALLOC_SCRATCH_BYTES))
        return fail(FFSRL_E_INVAL, "ffsrl_step_noalloc: this sim needs " + std::to_string(off) +
                                       " bytes of scratch but the static scratch array holds " +
                                       std::to_string(size_t(FFSRL_NOALLOC_SCRATCH_BYTES)) +
                                       " bytes (FFSRL_NOALLOC_SCRATCH_BYTES); use fewer envs per sim");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(sim->device, &base);
    if (rc) return rc;

    SimDev S = sim->S;
    S.x = reinterpret_cast<float*>(base + o_x);
    S.v = reinterpret_cast<float*>(base + o_v);
    S.pg = reinterpret_cast<float*>(base + o_p);
    S.xg = any_streaming ? reinterpret_cast<float4*>(base + o_xg) : nullptr;
    S.contacts = reinterpret_cast<int*>(base + o_c);
    int* env_ints = reinterpret_cast<int*>(base + o_env);
    S.t_step = env_ints;
    S.n_contacts = env_ints + n;
    S.l_prev = reinterpret_cast<float*>(env_ints + 2 * n);
    S.done_flag = reinterpret_cast<uint8_t*>(env_ints + 3 * n);
    S.lambda = lam_slots ? reinterpret_cast<float*>(base + o_lam) : nullptr;
    S.tool = tool_dev;
    // Step counters, contact counts, last distances and done flags start at zero.
    FFSRL_CUDA(cudaMemsetAsync(env_ints, 0, 3 * n * sizeof(int) + n, sim->stream));
    FFSRL_CUDA(launch_unpack(S, sim->d_pstart, x_dev, v_dev, sim->stream));
    FFSRL_CUDA(launch_all(sim, &S, actions_dev, nullptr, nullptr, nullptr, sim->stream));
    FFSRL_CUDA(launch_pack(S, sim->d_pstart, x_dev, v_dev, sim->stream));
    return FFSRL_OK;
}
