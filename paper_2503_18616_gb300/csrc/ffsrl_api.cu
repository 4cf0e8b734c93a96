// C ABI of the batched XPBD simulator: creation, reset, step, state access.
// Declarations and contracts are in include/ffsrl.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ffsrl.h"
#include "mesh_setup.h"
#include "xpbd_device.cuh"
#include "xpbd_launch.h"

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

// One launch group: envs of one mesh, resident in shared memory or not.
struct LaunchGroup {
    bool resident;
    size_t smem;
    int n;
    int* d_list;
};

}  // namespace

struct ffsrl_sim {
    int device = 0;
    cudaStream_t stream = nullptr;
    ffsrl_params params{};
    int n_env = 0, obs_dim = 0, block = 256;
    std::vector<HostMesh> meshes;
    std::vector<int> env_mesh, voff, pstart;
    long long stride = 0, total_verts = 0;
    std::vector<void*> dev_allocs;
    float* h_pinned = nullptr;  // staging for ffsrl_step_host
    float* d_stage = nullptr;
    SimDev S{};
    int* d_pstart = nullptr;
    std::vector<LaunchGroup> groups;
    int resident_envs = 0;

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
    if (b != 0 && b != 128 && b != 256 && b != 384 && b != 512 && b != 768 && b != 1024)
        return fail(FFSRL_E_INVAL, "block_threads must be 0, 128, 256, 384, 512, 768 or 1024");
    for (int k = 0; k < 5; ++k)
        if (p.reserved[k] != 0) return fail(FFSRL_E_INVAL, "reserved params must be zero");
    return FFSRL_OK;
}

int build_device(ffsrl_sim* s, const double* env_alpha) {
    const ffsrl_params& p = s->params;
    const int n_env = s->n_env;
    const double h = p.dt / p.substeps;

    // Per-mesh device tables in colour-major order.
    std::vector<MeshDev> md(s->meshes.size());
    for (size_t mi = 0; mi < s->meshes.size(); ++mi) {
        const HostMesh& m = s->meshes[mi];
        MeshDev& d = md[mi];
        d.V = m.V;
        d.Vp = round_up(m.V, 32);
        d.E = m.E;
        d.T = m.T;
        d.n_ecol = m.n_ecol;
        d.n_tcol = m.n_tcol;
        d.n_top = int(m.top.size());
        std::vector<uint32_t> eab(m.E);
        std::vector<float> ed(m.E);
        for (int q = 0; q < m.E; ++q) {
            const int e = m.eorder[q];
            eab[q] = uint32_t(m.edge[2 * e]) | (uint32_t(m.edge[2 * e + 1]) << 16);
            ed[q] = m.rest_len[e];
        }
        std::vector<uint2> tq(m.T);
        std::vector<float> tv(m.T);
        for (int q = 0; q < m.T; ++q) {
            const int t = m.torder[q];
            tq[q].x = uint32_t(m.tet[4 * t]) | (uint32_t(m.tet[4 * t + 1]) << 16);
            tq[q].y = uint32_t(m.tet[4 * t + 2]) | (uint32_t(m.tet[4 * t + 3]) << 16);
            tv[q] = m.V0[t];
        }
        std::vector<float4> rw(m.V);
        for (int i = 0; i < m.V; ++i)
            rw[i] = make_float4(m.rest[3 * i], m.rest[3 * i + 1], m.rest[3 * i + 2], m.inv_mass[i]);
        uint32_t* d_eab; float* d_ed; uint2* d_tq; float* d_tv; int* d_eo; int* d_to; float4* d_rw; int* d_top;
        FFSRL_CUDA(s->upload(&d_eab, eab.data(), eab.size()));
        FFSRL_CUDA(s->upload(&d_ed, ed.data(), ed.size()));
        FFSRL_CUDA(s->upload(&d_tq, tq.data(), tq.size()));
        FFSRL_CUDA(s->upload(&d_tv, tv.data(), tv.size()));
        FFSRL_CUDA(s->upload(&d_eo, m.ecol_off.data(), m.ecol_off.size()));
        FFSRL_CUDA(s->upload(&d_to, m.tcol_off.data(), m.tcol_off.size()));
        FFSRL_CUDA(s->upload(&d_rw, rw.data(), rw.size()));
        FFSRL_CUDA(s->upload(&d_top, m.top.data(), m.top.size()));
        d.edge_ab = d_eab; d.edge_d = d_ed; d.tet_abcd = d_tq; d.tet_V0 = d_tv;
        d.ecol_off = d_eo; d.tcol_off = d_to; d.rest_w = d_rw; d.top = d_top;
        // Tool box around the rest bounding box and tool start above the top face.
        for (int k = 0; k < 2; ++k) {
            d.box_lo[k] = m.bbmin[k] - p.tool_margin_xy;
            d.box_hi[k] = m.bbmax[k] + p.tool_margin_xy;
            d.tool_start[k] = (m.bbmin[k] + m.bbmax[k]) / 2;
        }
        d.box_lo[2] = m.bbmax[2] - p.tool_margin_below;
        d.box_hi[2] = m.bbmax[2] + p.tool_margin_above;
        d.tool_start[2] = m.bbmax[2] + p.tool_radius;
        d.min_len = float(1e-12 * m.extent);
    }
    MeshDev* d_md;
    FFSRL_CUDA(s->upload(&d_md, md.data(), md.size()));

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
        s->voff[e] = int(voff);
        s->pstart[e] = int(pst);
        voff += d.Vp;
        pst += d.V;
        if (p.iterations > 1) loff += d.E + d.T;
        if (voff > 0x7fffffffLL || pst > 0x7fffffffLL || loff > 0x7fffffffLL)
            return fail(FFSRL_E_INVAL, "too many vertices in total (more than 2^31 rows)");
    }
    s->stride = voff;
    s->total_verts = pst;
    EnvDev* d_ev;
    FFSRL_CUDA(s->upload(&d_ev, ev.data(), ev.size()));
    FFSRL_CUDA(s->upload(&s->d_pstart, s->pstart.data(), s->pstart.size()));

    SimDev& S = s->S;
    S.meshes = d_md;
    S.envs = d_ev;
    S.n_env = n_env;
    S.obs_dim = s->obs_dim;
    S.stride = s->stride;
    FFSRL_CUDA(s->alloc(&S.x, 3 * size_t(s->stride)));
    FFSRL_CUDA(s->alloc(&S.v, 3 * size_t(s->stride)));
    FFSRL_CUDA(cudaMemset(S.x, 0, 3 * size_t(s->stride) * sizeof(float)));
    FFSRL_CUDA(cudaMemset(S.v, 0, 3 * size_t(s->stride) * sizeof(float)));
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
    S.lambda = nullptr;
    if (p.iterations > 1) FFSRL_CUDA(s->alloc(&S.lambda, size_t(loff)));
    S.h = float(h);
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

    // Launch groups: per mesh, resident in shared memory when it fits.
    int max_optin = 0;
    FFSRL_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
    const size_t static_smem = 64;  // tool centre in the kernel's static shared memory
    bool any_streaming = false;
    for (size_t mi = 0; mi < md.size(); ++mi) {
        std::vector<int> list;
        for (int e = 0; e < n_env; ++e)
            if (s->env_mesh[e] == int(mi)) list.push_back(e);
        if (list.empty()) continue;
        LaunchGroup g;
        g.n = int(list.size());
        const size_t res = resident_smem_bytes(md[mi].Vp);
        g.resident = res + static_smem <= size_t(max_optin);
        g.smem = g.resident ? res : streaming_smem_bytes(md[mi].Vp);
        any_streaming |= !g.resident;
        if (g.resident) s->resident_envs += g.n;
        FFSRL_CUDA(s->upload(&g.d_list, list.data(), list.size()));
        s->groups.push_back(g);
    }
    S.xg = nullptr;
    S.pg = nullptr;
    if (any_streaming) {
        FFSRL_CUDA(s->alloc(&S.xg, size_t(s->stride)));
        FFSRL_CUDA(s->alloc(&S.pg, 3 * size_t(s->stride)));
    }

    // Pinned host staging and device staging for ffsrl_step_host.
    const size_t stage = size_t(n_env) * (3 + s->obs_dim + 1) + (size_t(n_env) + 3) / 4;
    FFSRL_CUDA(cudaMallocHost(&s->h_pinned, stage * sizeof(float)));
    FFSRL_CUDA(s->alloc(&s->d_stage, stage));
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
    s->block = params->block_threads ? params->block_threads : 256;
    s->meshes.resize(n_meshes);
    for (int i = 0; i < n_meshes; ++i) {
        std::string err;
        rc = build_host_mesh(meshes[i].n_verts, meshes[i].n_tets, meshes[i].rest_pos, meshes[i].inv_mass,
                             meshes[i].tets, s->meshes[i], err);
        if (rc) {
            delete s;
            return fail(rc, "mesh " + std::to_string(i) + ": " + err);
        }
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
        cudaError_t e = launch_reset(s->S, nullptr, 0ull, s->stream);
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

int ffsrl_step(ffsrl_sim* sim, const float* actions_dev, float* obs_dev, float* reward_dev,
               uint8_t* done_dev) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    for (const LaunchGroup& g : sim->groups)
        FFSRL_CUDA(launch_step(sim->S, g.resident, sim->block, g.d_list, g.n, g.smem, sim->stream,
                               actions_dev, obs_dev, reward_dev, done_dev));
    return FFSRL_OK;
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
    if (actions_host) {
        std::memcpy(h_act, actions_host, 3 * n * sizeof(float));
        FFSRL_CUDA(cudaMemcpyAsync(d_act, h_act, 3 * n * sizeof(float), cudaMemcpyHostToDevice, sim->stream));
    }
    int rc = ffsrl_step(sim, actions_host ? d_act : nullptr, obs_host ? d_obs : nullptr,
                        reward_host ? d_rew : nullptr, done_host ? d_done : nullptr);
    if (rc) return rc;
    if (obs_host)
        FFSRL_CUDA(cudaMemcpyAsync(h_obs, d_obs, od * n * sizeof(float), cudaMemcpyDeviceToHost, sim->stream));
    if (reward_host)
        FFSRL_CUDA(cudaMemcpyAsync(h_rew, d_rew, n * sizeof(float), cudaMemcpyDeviceToHost, sim->stream));
    if (done_host)
        FFSRL_CUDA(cudaMemcpyAsync(h_done, d_done, n, cudaMemcpyDeviceToHost, sim->stream));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    if (obs_host) std::memcpy(obs_host, h_obs, od * n * sizeof(float));
    if (reward_host) std::memcpy(reward_host, h_rew, n * sizeof(float));
    if (done_host) std::memcpy(done_host, h_done, n);
    return FFSRL_OK;
}

int ffsrl_sync(ffsrl_sim* sim) {
    if (!sim) return fail(FFSRL_E_INVAL, "sim is NULL");
    FFSRL_CUDA(cudaSetDevice(sim->device));
    FFSRL_CUDA(cudaStreamSynchronize(sim->stream));
    std::vector<int> err(sim->n_env);
    FFSRL_CUDA(cudaMemcpy(err.data(), sim->S.err, err.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int first = -1;
    for (int e = 0; e < sim->n_env; ++e)
        if (err[e] && first < 0) first = e;
    if (first >= 0) {
        FFSRL_CUDA(cudaMemset(sim->S.err, 0, err.size() * sizeof(int)));
        return fail(FFSRL_E_NAN, "non-finite positions in env " + std::to_string(first));
    }
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
    out->block_threads = sim->block;
    out->resident_envs = sim->resident_envs;
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
