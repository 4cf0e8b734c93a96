// Host-side constraint-table construction for the XPBD simulator.
//
// Everything the paper computes "before the simulation loop" (FF-SRL,
// arXiv 2503.18616, Sec. III-A): edge list and rest distances d_ab (Eq. 1),
// oriented tets and rest volumes V0 (Eq. 2), plus the graph colouring that
// lets constraints of one colour be projected in parallel, the colour-major
// constraint order, and the top-face vertex list used for observations.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace ffsrl {

struct HostMesh {
    int V = 0, T = 0, E = 0;
    std::vector<float> rest;        // [V*3], float32 rest positions
    std::vector<float> inv_mass;    // [V]
    std::vector<int32_t> tet;       // [T*4] oriented (positive rest volume)
    std::vector<int32_t> flipped;   // [T]
    std::vector<float> V0;          // [T]
    std::vector<int32_t> edge;      // [E*2], (min, max), ascending
    std::vector<float> rest_len;    // [E]
    int n_ecol = 0, n_tcol = 0;
    std::vector<int32_t> ecolor, tcolor;      // per constraint
    std::vector<int32_t> eorder, torder;      // colour-major position -> constraint
    std::vector<int32_t> ecol_off, tcol_off;  // [n_col + 1]
    std::vector<int32_t> top;                 // ascending ids with z == max z
    // surface faces (faces of exactly one tet with a free vertex), ascending
    // by sorted vertex triple, for the grasper collision; colour-major order
    int F = 0, n_fcol = 0;
    std::vector<int32_t> face;                // [F][3] ascending vertex ids
    std::vector<int32_t> fopp;                // [F] fourth vertex of the face's tet
    std::vector<int32_t> fcolor, forder, fcol_off;
    // objects (connected components of the tets, numbered by lowest vertex)
    // and tissue connections: vertex, then a surface face of a lower object
    // whose centroid is nearest at rest within the connection radius
    int n_obj = 0, C = 0, n_ccol = 0;
    std::vector<int32_t> obj;                 // [V]
    std::vector<int32_t> conn;                // [C][4]
    std::vector<float> conn_d0;               // [C] rest distance, vertex to centroid
    std::vector<int32_t> ccolor, corder, ccol_off;
    double bbmin[3] = {0, 0, 0}, bbmax[3] = {0, 0, 0};
    double extent = 0;
    // Order of each tet's vertices in the GPU's records: an even permutation
    // of tet[4t .. 4t+3] (index into kEvenPerm; empty = all identity). The
    // signed volume, hence V0, is unchanged; the bank-aware schedule chooses
    // them and every schedule of the mesh then uses the same order.
    std::vector<uint8_t> tet_rot;
};

// The 12 even permutations of four positions (row 0 the identity): record
// position k holds tet vertex kEvenPerm[r][k].
extern const int kEvenPerm[12][4];

// Returns 0 or a negative FFSRL_E_* code with a message in err.
// conn_radius > 0 adds tissue connections between the mesh's objects.
int build_host_mesh(int V, int T, const double* rest, const double* inv_mass,
                    const int32_t* tets, HostMesh& out, std::string& err, double conn_radius = 0.0);

// Objects and tissue connections of a mesh whose faces are built (rest: the
// positions as given); called by build_host_mesh.
int build_connections(HostMesh& m, const double* rest, double conn_radius, std::string& err);

// Execution schedule of one mesh on the GPU: vertex -> shared-memory slot map
// and the constraint stream in phases (edge phases, then tet phases, then
// connection phases), each phase a 16-byte aligned segment of records. The
// phases are the colours, or (permuted schedules) a refinement of the
// colouring into phases of whole multiples of kPhaseUnit constraints that
// keeps, at every vertex, the colour order of the constraints containing it,
// and therefore gives the same bits.
struct Schedule {
    std::vector<uint16_t> slot_of, vert_of;  // [V]
    std::vector<unsigned char> stream;       // records
    std::vector<int32_t> segs;               // [n_seg][4]: byte offset, bytes, count, first constraint
    int ring_bytes = 0;                      // largest segment
    int parts = 1;                           // segments per colour (one per cluster CTA)
    int part_slots = 0;                      // slots per part (multiple of 32)
    int n_ephase = 0, n_tphase = 0, n_cphase = 0;   // phases per family
    std::vector<uint8_t> tet_rot;            // [T] the vertex orders the tet records use
    // [F][4] surface-face records for the grasper, colour-major like
    // HostMesh::forder (same colour sizes): slot(a) | slot(b) << 16,
    // slot(c) | slot(opposite vertex) << 16, 0, 0; with the permutation each
    // colour's faces are grouped in 8s by bank groups of a, b and c
    std::vector<uint32_t> frec;
};

constexpr int kPhaseUnit = 256;              // threads per env of the common step configuration
// Refined phases (capped at 4 KB of records) are built for meshes small enough
// that four such CTAs fit an SM; larger meshes run more threads per env (or a
// cluster) and keep the colours, where extra phase barriers would cost more
// than the thread rounds they save.
constexpr int kPhaseMaxVerts = 2944;

// Builds the schedule. Slots are a fixed permutation inside each aligned
// block of 32 vertices (seeded by `seed`); inside each phase the records are
// grouped so that the 8 records of every aligned group of 8 use distinct
// slot residues modulo 8 in each vertex position where possible (distinct
// shared-memory bank groups for 16-byte accesses). With `permute` (one part,
// at most kPhaseMaxVerts vertices) the phases are the refinement described
// above, else the colours. None of these
// choices changes the result: a phase's constraints touch disjoint vertices
// and every vertex sees its constraints in colour order.
// With parts > 1 the slots are split into `parts` ranges of part_slots slots
// (one per CTA of a thread-block cluster) and every phase into `parts`
// segments, segment r holding the records whose first vertex lies in range r
// (segments ordered phase-major, part-minor).
void build_schedule(const HostMesh& m, uint64_t seed, bool permute, Schedule& out, int parts = 1);

}  // namespace ffsrl
