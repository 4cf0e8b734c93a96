// Device-side data layout of the batched XPBD simulator (sm_103a).
//
// HBM layout (one allocation per array, all envs concatenated, Sec. III-B of
// FF-SRL, arXiv 2503.18616):
//   positions / velocities: structure of arrays, x[k * stride + voff_e + i] for
//     component k, env e, vertex i; voff_e is a multiple of 32 vertices so every
//     env starts on a 128-byte boundary.
//   constraint stream: per distinct mesh, one byte stream holding every colour
//     (edge colours, then tet colours) as a 16-byte aligned segment of records.
//     Edge record (8 B): slot(a) | slot(b) << 16, rest length. Tet record (16 B):
//     slot(a) | slot(b) << 16, slot(c) | slot(d) << 16, rest volume, unused.
//     Vertex "slots" are the shared-memory rows of the vertices: a fixed
//     permutation inside each aligned block of 32 vertices, chosen with the
//     order of records inside each colour so that the 8 lanes of each
//     shared-memory access phase hit distinct bank groups. Records of one
//     colour touch disjoint vertices, so their order does not change results.
//   per-env scalars: tool centre (float64), last distance, step count, seed,
//     target vertex, observed vertex ids, contact list, error flags.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ffsrl {

struct MeshDev {
    int V, Vp, E, T;
    int n_ecol, n_tcol, n_top, n_seg;  // segments: edge colours, tet colours, connection colours
    int ring_bytes;                   // largest segment in bytes (one ring stage)
    int n_dseg;                       // edge and tet segments (the rest are tissue connections)
    const unsigned char* recs;        // constraint stream
    // the same stream with every slot field holding the slot's byte offset
    // (slot x 16), for meshes of at most 4096 slots in one part (else null):
    // a record then addresses shared memory without a shift
    const unsigned char* recs16;
    const int4* segs;                 // [n_seg] {byte offset, bytes, count, first constraint}
    const uint16_t* slot_of;          // [V] shared-memory slot of each vertex
    const uint16_t* vert_of;          // [V] vertex of each slot
    const float4* rest_w;             // [V] rest position and inverse mass (vertex order)
    const int* top;                   // [n_top] top-face vertex ids
    const int* nbr_off;               // [V + 1] 1-ring of each vertex (vertex order, CSR)
    const int* nbr;                   // [2E]
    // 1-ring of each slot in slot terms (same neighbour order as nbr): the
    // 48-byte record of slot s, snbr[3 s .. 3 s + 2], holds 24 uint16 fields:
    // its degree, then its neighbour slots (at most 23; a mesh with a larger
    // 1-ring has no records: snbr is null).
    const uint4* snbr;
    const float4* rest_s;             // [V] rest position and inverse mass (slot order)
    int max_deg;                      // largest vertex degree
    int tile_reach;                   // largest |s / 128 - j / 128| over slots s and their 1-ring slots j
    int parts;                        // segments per colour (CTAs of a cluster holding one env)
    int part_slots;                   // slots per part, a multiple of 32 (parts > 1)
    const float* inv_ncons;           // [V] 1 / (constraints containing the slot's vertex), slot order
    // surface faces for the grasper: record {slot a | slot b << 16, slot c | slot of the
    // opposite tet vertex << 16, 0, 0} in colour-major order, colour offsets
    int F, n_fcol;
    const uint4* frec;
    const int* fcol_off;              // [n_fcol + 1]
    float rcm[3];                     // remote centre of motion of the grasper
    int first_free_tile;              // 128-slot tiles before it hold pinned vertices only
    const uint2* erec;                // [E] edge records of the stream, unpadded, stream order
    const uint4* trec;                // [T] tet records of the stream, unpadded, stream order
    double box_lo[3], box_hi[3], tool_start[3];
    float min_len2;                   // edges with |x_ab|^2 below this are skipped
    int pad1;
};

struct EnvDev {
    int mesh;       // index into the mesh table
    int voff;       // first padded vertex row of this env
    float alpha_d;  // edge compliance / h^2 (alpha tilde of XPBD)
    int loff;       // first lambda slot of this env (iterations > 1)
    unsigned long long gid;  // global env id of the counter-based draws (the env index by default)
};

// Error bits in SimDev::err.
constexpr int kErrNonFinite = 1;
constexpr int kErrTimeout = 2;

struct SimDev {
    const MeshDev* meshes;
    const EnvDev* envs;
    int n_env;
    int obs_dim;
    long long stride;         // padded vertex rows over all envs
    float* x;                 // [3][stride] vertex order
    float* v;                 // [3][stride]
    double* tool;             // [n_env][3]
    float* l_prev;            // [n_env]
    int* t_step;              // [n_env]
    unsigned long long* seed; // [n_env]
    int* obs_ids;             // [n_env][n_obs]
    int* target;              // [n_env]
    int* n_contacts;          // [n_env]
    int* contacts;            // [stride]: env e's list at voff_e
    int* err;                 // [n_env] kErr* bits
    float* lambda;            // multipliers carried across iterations (iterations > 1)
    uint8_t* done_flag;       // [n_env] done of the env's last step (auto-reset)
    unsigned long long* seed0;  // [n_env] seed given to reset
    int* episode;             // [n_env] episodes started by auto-reset since then
    float4* xg;               // [stride] working positions (slot order) of envs not resident in SMEM
    float* pg;                // [3][stride] substep-start positions (slot order)
    float h, inv_h, gx, gy, gz;
    float alpha_v;            // volume compliance / h^2
    float radius;
    double action_scale;
    int substeps, iterations, n_obs, max_steps;
    double w_l, w_d, w_s, success_dist;
    int tool_model;           // 0 sphere, 1 grasper
    float shaft_radius, clamp_length, clamp_radius;
    float clamp_angle0;       // clamp opening at reset (radians)
    float2 clamp_cs0;         // its cosine and sine
    float grasp_radius;
    float* clamp_angle;       // [n_env] current clamp opening (radians)
    float2* clamp_cs;         // [n_env] its cosine and sine (kept beside it, so the step needs no trigonometry)
    int* grasp_v;             // [n_env] grasped vertex or -1
    float* grasp_d0;          // [n_env] its grasp-time distance to the dragging point
};

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the n-th output of the
// generator started at `state` is the output mix of state + (n + 1) * gamma.
__host__ __device__ __forceinline__ unsigned long long splitmix64_nth(unsigned long long state,
                                                                      unsigned long long n) {
    unsigned long long z = state + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Stream of env `env` for draw family `family` (0 actions, 1 observed vertices, 2 target).
__host__ __device__ __forceinline__ unsigned long long env_stream(unsigned long long seed,
                                                                  unsigned long long env,
                                                                  unsigned family) {
    return splitmix64_nth(seed, 4ull * env + family);
}

// Top 24 bits as a number in [-1, 1): exact in float32 and float64.
__host__ __device__ __forceinline__ double to_unit_pm1(unsigned long long r) {
    return 2.0 * (double)(r >> 40) * (1.0 / 16777216.0) - 1.0;
}

}  // namespace ffsrl
