/*
 * Plain, sequential CPU oracle for the FF-SRL batched XPBD step
 * (Dall'Alba et al., "FF-SRL: High Performance GPU-Based Surgical Simulation
 * For Robot Learning", arXiv 2503.18616).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark are the only code allowed to load this
 * library. The simulator library never links, loads or calls it, and the two
 * share no source, header, table or helper. Everything here is written for a
 * reader who checks it against the paper by eye: one environment at a time,
 * one constraint at a time, in the order the method defines, no blocking,
 * fusion or reordering.
 *
 * Precision: REAL is double (liboracle_f64). The same file compiled with
 * -DREAL=float (liboracle_f32) exists only to measure the FP32 rounding floor.
 *
 * What each part follows (section numbers of the paper):
 *   - simulation loop ............ Algorithm 1 (Sec. III-A), with the readings below
 *   - edge-distance constraint ... Eq. 1, XPBD compliance form (MacklinXPBD2016,
 *                                  the XPBD paper the method builds on, Sec. III-A)
 *   - tet-volume constraint ...... Eqs. 2-3, with the corrected gradient assignment
 *   - tool collision ............. Sec. III-A "Collisions", sphere proxy vs vertices
 *   - reward / termination ....... Sec. IV (reward R = w_l l + w_d d + w_s s), Sec. III-B
 *   - substepping ................ Sec. III-A (n substeps x 1 iteration)
 *
 * Readings where the paper is silent, garbled or differs from the default
 * configuration built here (each is also listed in the design notes of the
 * repository):
 *   R1  Eq. 2 assigns the cross products to the wrong vertices and flips the
 *       sign of the d term. Used here: g_b = x_ca x x_da / 6,
 *       g_c = x_da x x_ba / 6, g_d = x_ba x x_ca / 6, g_a = -(g_b+g_c+g_d),
 *       the exact gradient of C = (x_ba x x_ca).x_da / 6 - V0.
 *   R2  Stiffness k in [0,1] is replaced by XPBD compliance: alpha~ = alpha/h^2,
 *       dlambda = (-C - alpha~ lambda) / (sum_i w_i |g_i|^2 + alpha~),
 *       dx_i = w_i dlambda g_i; lambda reset to 0 at the start of every substep.
 *   R3  Eq. 3's denominator gains the inverse masses w_i (needed for pins).
 *   R4  Constraints run as graph-coloured Gauss-Seidel: all distance colours,
 *       then all volume colours; inside a colour no two constraints share a
 *       vertex, so visiting order inside a colour does not change the result.
 *       Colouring is greedy first-fit: edges in ascending (min,max) order,
 *       tets in input order, the two families coloured separately.
 *   R5  Collision runs once per substep, after the constraint iterations and
 *       before the velocity update.
 *   R6  Sphere test is strict (|d| < r); |d| = 0 pushes along +z; pinned
 *       vertices (w = 0) never move; the tool is kinematic.
 *   R7  The tool moves once per step, at its start, then stays put for the
 *       substeps; it is clamped to a box around the rest bounding box.
 *   R8  Degenerate constraints are skipped: zero denominator, or an edge
 *       shorter than 1e-12 x extent. A tet with negative rest volume has its
 *       last two vertices swapped at setup.
 *   R9  Counter-based RNG: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).
 *   R10 The paper's own GPU scheme (Sec. III-A) as an option: Jacobi
 *       iterations in which every constraint steps from the iteration's start
 *       positions and each vertex moves by the sum of its corrections divided
 *       by the number of constraints (distance and volume) that contain it;
 *       multipliers as in R2.
 *   R11 Optional auto-reset: an env whose step reported done starts episode
 *       k+1 at its next step, from the rest state with the draws of seed
 *       splitmix64_nth(seed, 2^40 + k+1) (seed = the one given to reset; the
 *       actions of the episode use that seed too).
 *   R12 Optional grasper tool (Sec. III-A "Surgical tool model"): the tool
 *       point c (moved by the actions as in R7) is the end of the shaft; the
 *       shaft runs from the remote centre of motion (above the centre of the
 *       top face) to c, so it always passes through that centre; two clamps
 *       leave c at +-alpha from the shaft axis in the plane of the axis and
 *       world x. Each part is a capsule (segment and radius). The tool starts
 *       with the clamp tips touching the centre of the top face.
 *   R13 Grasper collision (Sec. III-A "Collisions"): once per substep after
 *       the iterations, the surface faces (faces of exactly one tet with a
 *       free vertex) are visited colour by colour (first-fit, ascending
 *       triples); each face against the shaft, then the clamps: with p the
 *       face's closest point to the capsule axis (barycentric b) and q the
 *       axis point, if |p - q| < r the face is pushed along n = (p-q)/|p-q| by
 *       a PBD step of stiffness 1: x_j -= w_j b_j (|p-q| - r) n / sum w b^2.
 *       If the axis crosses the face, n points from the axis to the face's
 *       centroid (or, if that is on the axis too, into the tissue).
 *   R14 The per-element local optimisation the paper follows finds the
 *       face's point of least capsule distance; here that point is computed
 *       exactly (segment-triangle closest points).
 *   R15 Grasping (Sec. III-A, dragging): the dragging point is the end of the
 *       closed clamps, clamp_length beyond the tool point along the shaft
 *       axis. At the start of a step, clamps closed below 3 degrees take the
 *       free vertex nearest to it within grasp_radius (ties: lower id; kept
 *       until the clamps open to 3 degrees or more); each substep, after the
 *       iterations and before the face collision, a distance constraint of
 *       stiffness 1 keeps that vertex at its grasp-time distance from the
 *       dragging point (the tool is kinematic: only the vertex moves).
 *   R16 Tissue connections (Sec. III-A): a mesh may hold several objects
 *       (the connected components of its tets, numbered by their lowest
 *       vertex). Every vertex of a surface face (R13) of object o connects to
 *       the surface face of a lower-numbered object whose centroid is nearest
 *       at rest (ties: the first face in ascending triple order), if that
 *       distance is at most conn_radius. The constraint keeps the distance
 *       from the vertex to the face's centroid at its rest value:
 *       C = |x_v - (x_a + x_b + x_c) / 3| - d0, gradients n at v and -n/3 at
 *       a, b, c; a distance constraint with the distance compliance (R2).
 *       Connections are coloured first-fit in vertex order and projected in
 *       every iteration after the volume colours; the selection is computed
 *       in double from the input rest positions in either build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#endif

#define ORC_OK 0
#define ORC_E_INVAL (-1)
#define ORC_E_OOM (-3)
#define ORC_E_DEGENERATE (-4)
#define ORC_MAX_COLORS 256

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers (R9).                                        */
/* ------------------------------------------------------------------------ */

static const uint64_t ORC_GOLDEN_GAMMA = 0x9E3779B97F4A7C15ULL;

/* SplitMix64 output function applied to one state word. */
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The n-th (0-based) output of SplitMix64 started from state `state`. */
uint64_t orc_sm64(uint64_t state, uint64_t n) {
    return orc_mix64(state + (n + 1) * ORC_GOLDEN_GAMMA);
}

/* Per-environment stream: domain 0 = actions, 1 = observation sample,
 * 2 = target vertex. */
uint64_t orc_stream(uint64_t seed, uint64_t env, uint32_t domain) {
    return orc_sm64(seed, 4 * env + domain);
}

/* Top 24 bits of r as a uniform number in [-1, 1). */
double orc_uniform_pm1(uint64_t r) {
    double u = (double)(r >> 40) * (1.0 / 16777216.0);
    return 2.0 * u - 1.0;
}

/* Action component `axis` of environment `env` at its step `t` since reset. */
double orc_action(uint64_t seed, uint64_t env, uint64_t t, int axis) {
    return orc_uniform_pm1(orc_sm64(orc_stream(seed, env, 0), 3 * t + (uint64_t)axis));
}

/* Floyd's sampling of k distinct indices from [0, n), sorted ascending. */
int orc_sample_indices(uint64_t seed, uint64_t env, int n, int k, int* out) {
    if (k < 0 || k > n) return ORC_E_INVAL;
    uint64_t st = orc_stream(seed, env, 1);
    int m = 0;
    for (int j = n - k; j < n; ++j) {
        uint64_t r = orc_sm64(st, (uint64_t)j);
        int t = (int)(r % (uint64_t)(j + 1));
        int taken = 0;
        for (int q = 0; q < m; ++q)
            if (out[q] == t) taken = 1;
        out[m++] = taken ? j : t;
    }
    for (int a = 1; a < m; ++a) { /* insertion sort */
        int key = out[a], b = a - 1;
        while (b >= 0 && out[b] > key) { out[b + 1] = out[b]; --b; }
        out[b + 1] = key;
    }
    return ORC_OK;
}

int orc_target_index(uint64_t seed, uint64_t env, int n) {
    return (int)(orc_sm64(orc_stream(seed, env, 2), 0) % (uint64_t)n);
}

/* ------------------------------------------------------------------------ */
/* Small vector helpers.                                                     */
/* ------------------------------------------------------------------------ */

static void vsub(const REAL* a, const REAL* b, REAL* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static void vcross(const REAL* a, const REAL* b, REAL* o) {
    REAL t0 = a[1] * b[2] - a[2] * b[1];
    REAL t1 = a[2] * b[0] - a[0] * b[2];
    REAL t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static REAL vdot(const REAL* a, const REAL* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static REAL vnorm(const REAL* a) { return sqrt(vdot(a, a)); }

/* Signed tet volume (x_ba x x_ca) . x_da / 6 (the C^v definition, Sec. III-A). */
static REAL tet_volume(const REAL* xa, const REAL* xb, const REAL* xc, const REAL* xd) {
    REAL ba[3], ca[3], da[3], n[3];
    vsub(xb, xa, ba); vsub(xc, xa, ca); vsub(xd, xa, da);
    vcross(ba, ca, n);
    return vdot(n, da) / 6;
}

/* ------------------------------------------------------------------------ */
/* Mesh setup (Sec. III-A: vertices, edges, tets; rest distance and rest     */
/* volume computed before the loop; R4 colouring, R8 orientation).           */
/* ------------------------------------------------------------------------ */

typedef struct orc_mesh {
    int V, T, E;
    REAL* rest;     /* [V][3] */
    REAL* w;        /* [V] inverse mass, 0 = pinned */
    int* tet;       /* [T][4] oriented */
    int* flipped;   /* [T] 1 if vertices 2 and 3 were swapped */
    REAL* V0;       /* [T] rest volume (> 0) */
    int* edge;      /* [E][2], edge[0] < edge[1], ascending */
    REAL* d;        /* [E] rest length */
    int n_ecol, n_tcol;
    int* ecolor;    /* [E] */
    int* tcolor;    /* [T] */
    int* eorder;    /* [E] colour-major order: position -> edge id */
    int* torder;    /* [T] */
    int* ecol_off;  /* [n_ecol + 1] */
    int* tcol_off;  /* [n_tcol + 1] */
    int n_top;
    int* top;       /* ascending ids of vertices with z == max z */
    REAL bbmin[3], bbmax[3];
    REAL extent;    /* max side of the rest bounding box */
    /* surface faces (faces of exactly one tet) with at least one free vertex,
     * ascending by sorted vertex triple, for the grasper collision (R13) */
    int F;
    int* face;      /* [F][3] ascending vertex ids */
    int* fopp;      /* [F] the fourth vertex of the face's tet (outward normal points away from it) */
    int n_fcol;
    int* fcolor;    /* [F] first-fit colour */
    int* forder;    /* [F] colour-major order */
    int* fcol_off;  /* [n_fcol + 1] */
    /* tissue connections (R16) */
    int n_obj;
    int* obj;       /* [V] object (connected component) of each vertex */
    int C;
    int* conn;      /* [C][4] vertex, then the face's ascending triple */
    REAL* cd0;      /* [C] rest distance from the vertex to the face's centroid */
    int n_ccol;
    int* ccolor;    /* [C] first-fit colour */
    int* corder;    /* [C] colour-major order */
    int* ccol_off;  /* [n_ccol + 1] */
} orc_mesh;

void orc_mesh_destroy(orc_mesh* m) {
    if (!m) return;
    free(m->rest); free(m->w); free(m->tet); free(m->flipped); free(m->V0);
    free(m->edge); free(m->d); free(m->ecolor); free(m->tcolor);
    free(m->eorder); free(m->torder); free(m->ecol_off); free(m->tcol_off);
    free(m->top); free(m->face); free(m->fopp); free(m->fcolor); free(m->forder); free(m->fcol_off);
    free(m->obj); free(m->conn); free(m->cd0); free(m->ccolor); free(m->corder); free(m->ccol_off);
    free(m);
}

static int cmp_triple(const void* pa, const void* pb) {
    const int* a = (const int*)pa;
    const int* b = (const int*)pb;
    for (int k = 0; k < 3; ++k)
        if (a[k] != b[k]) return a[k] < b[k] ? -1 : 1;
    return 0;
}

static int cmp_pair(const void* pa, const void* pb) {
    const int* a = (const int*)pa; const int* b = (const int*)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

/* Greedy first-fit colouring: constraint i (visited in index order) takes the
 * smallest colour used by no earlier constraint that shares a vertex with it.
 * used[v][c] marks colour c as taken at vertex v. */
static int color_first_fit(int n, int arity, const int* cons, int V, int* color, int* n_colors) {
    unsigned char* used = (unsigned char*)calloc((size_t)V * ORC_MAX_COLORS, 1);
    if (!used) return ORC_E_OOM;
    int nc = 0;
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (;;) {
            int clash = 0;
            for (int k = 0; k < arity; ++k)
                if (used[(size_t)cons[i * arity + k] * ORC_MAX_COLORS + c]) clash = 1;
            if (!clash) break;
            ++c;
            if (c >= ORC_MAX_COLORS) { free(used); return ORC_E_INVAL; }
        }
        color[i] = c;
        for (int k = 0; k < arity; ++k) used[(size_t)cons[i * arity + k] * ORC_MAX_COLORS + c] = 1;
        if (c + 1 > nc) nc = c + 1;
    }
    free(used);
    *n_colors = nc;
    return ORC_OK;
}

/* Stable colour-major order: constraints sorted by (colour, index). */
static void color_major(int n, const int* color, int nc, int* order, int* off) {
    int p = 0;
    for (int c = 0; c < nc; ++c) {
        off[c] = p;
        for (int i = 0; i < n; ++i)
            if (color[i] == c) order[p++] = i;
    }
    off[nc] = p;
}

/* Objects and tissue connections (R16), from the input rest positions in
 * double. Returns ORC_OK or an error code. */
static int build_connections(orc_mesh* m, const double* rest, double conn_radius) {
    const int V = m->V;
    /* objects: connected components of the tets, labelled from the lowest
     * unlabelled vertex upwards (so object ids follow their lowest vertex) */
    m->obj = (int*)malloc(sizeof(int) * V);
    int* vt_off = (int*)calloc(V + 1, sizeof(int));
    int* vt = (int*)malloc(sizeof(int) * (4 * m->T > 0 ? 4 * m->T : 1));
    int* stack = (int*)malloc(sizeof(int) * V);
    for (int t = 0; t < m->T; ++t)
        for (int k = 0; k < 4; ++k) vt_off[m->tet[4 * t + k] + 1]++;
    for (int i = 0; i < V; ++i) vt_off[i + 1] += vt_off[i];
    int* fill = (int*)malloc(sizeof(int) * (V > 0 ? V : 1));
    for (int i = 0; i < V; ++i) fill[i] = vt_off[i];
    for (int t = 0; t < m->T; ++t)
        for (int k = 0; k < 4; ++k) vt[fill[m->tet[4 * t + k]]++] = t;
    for (int i = 0; i < V; ++i) m->obj[i] = -1;
    m->n_obj = 0;
    for (int i = 0; i < V; ++i) {
        if (m->obj[i] >= 0) continue;
        int top = 0;
        stack[top++] = i;
        m->obj[i] = m->n_obj;
        while (top > 0) {
            const int u = stack[--top];
            for (int q = vt_off[u]; q < vt_off[u + 1]; ++q)
                for (int k = 0; k < 4; ++k) {
                    const int x = m->tet[4 * vt[q] + k];
                    if (m->obj[x] < 0) { m->obj[x] = m->n_obj; stack[top++] = x; }
                }
        }
        m->n_obj++;
    }
    free(vt_off); free(vt); free(stack); free(fill);
    /* connections: each vertex of a surface face, in ascending order */
    m->conn = (int*)malloc(sizeof(int) * 4 * (V > 0 ? V : 1));
    m->cd0 = (REAL*)malloc(sizeof(REAL) * (V > 0 ? V : 1));
    m->C = 0;
    unsigned char* on_face = (unsigned char*)calloc(V > 0 ? V : 1, 1);
    for (int f = 0; f < m->F; ++f)
        for (int k = 0; k < 3; ++k) on_face[m->face[3 * f + k]] = 1;
    if (conn_radius > 0)
        for (int i = 0; i < V; ++i) {
            if (!on_face[i]) continue;
            int best = -1;
            double bd2 = 0;
            for (int f = 0; f < m->F; ++f) {
                const int* fv = &m->face[3 * f];
                if (!(m->obj[fv[0]] < m->obj[i])) continue;
                double d2 = 0;
                for (int k = 0; k < 3; ++k) {
                    const double centroid = (rest[3 * fv[0] + k] + rest[3 * fv[1] + k] + rest[3 * fv[2] + k]) / 3.0;
                    const double dk = rest[3 * i + k] - centroid;
                    d2 += dk * dk;
                }
                if (best < 0 || d2 < bd2) { best = f; bd2 = d2; }
            }
            if (best < 0 || !(sqrt(bd2) <= conn_radius)) continue;
            int* c = &m->conn[4 * m->C];
            c[0] = i;
            c[1] = m->face[3 * best]; c[2] = m->face[3 * best + 1]; c[3] = m->face[3 * best + 2];
            m->cd0[m->C] = (REAL)sqrt(bd2);
            m->C++;
        }
    free(on_face);
    m->ccolor = (int*)malloc(sizeof(int) * (m->C > 0 ? m->C : 1));
    m->corder = (int*)malloc(sizeof(int) * (m->C > 0 ? m->C : 1));
    int rc = color_first_fit(m->C, 4, m->conn, V, m->ccolor, &m->n_ccol);
    if (rc != ORC_OK) return rc;
    m->ccol_off = (int*)malloc(sizeof(int) * (m->n_ccol + 1));
    color_major(m->C, m->ccolor, m->n_ccol, m->corder, m->ccol_off);
    return ORC_OK;
}

/* Builds the mesh tables. If edges_in is given (n_edges_in pairs), it replaces
 * the edge extraction from tets (used only by pins with a single constraint).
 * conn_radius > 0 adds the tissue connections of R16. Returns NULL and sets
 * *err on failure. */
orc_mesh* orc_mesh_create(int V, const double* rest, const double* w, int T, const int* tets,
                          int n_edges_in, const int* edges_in, double conn_radius, int* err) {
    *err = ORC_E_INVAL;
    if (V <= 0 || T < 0 || (T == 0 && !edges_in)) return NULL;
    orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
    if (!m) { *err = ORC_E_OOM; return NULL; }
    m->V = V; m->T = T;
    m->rest = (REAL*)malloc(sizeof(REAL) * 3 * V);
    m->w = (REAL*)malloc(sizeof(REAL) * V);
    m->tet = (int*)malloc(sizeof(int) * 4 * (T > 0 ? T : 1));
    m->flipped = (int*)calloc(T > 0 ? T : 1, sizeof(int));
    m->V0 = (REAL*)malloc(sizeof(REAL) * (T > 0 ? T : 1));
    for (int i = 0; i < 3 * V; ++i) m->rest[i] = (REAL)rest[i];
    for (int i = 0; i < V; ++i) {
        m->w[i] = (REAL)w[i];
        if (!(w[i] >= 0)) { orc_mesh_destroy(m); return NULL; }
    }
    /* bounding box and extent */
    for (int k = 0; k < 3; ++k) { m->bbmin[k] = m->rest[k]; m->bbmax[k] = m->rest[k]; }
    for (int i = 0; i < V; ++i)
        for (int k = 0; k < 3; ++k) {
            if (m->rest[3 * i + k] < m->bbmin[k]) m->bbmin[k] = m->rest[3 * i + k];
            if (m->rest[3 * i + k] > m->bbmax[k]) m->bbmax[k] = m->rest[3 * i + k];
        }
    m->extent = 0;
    for (int k = 0; k < 3; ++k)
        if (m->bbmax[k] - m->bbmin[k] > m->extent) m->extent = m->bbmax[k] - m->bbmin[k];
    /* tets: validate, orient (R8), rest volume */
    for (int t = 0; t < T; ++t) {
        int q[4];
        for (int k = 0; k < 4; ++k) {
            q[k] = tets[4 * t + k];
            if (q[k] < 0 || q[k] >= V) { orc_mesh_destroy(m); return NULL; }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (q[a] == q[b]) { orc_mesh_destroy(m); return NULL; }
        REAL vol = tet_volume(&m->rest[3 * q[0]], &m->rest[3 * q[1]], &m->rest[3 * q[2]], &m->rest[3 * q[3]]);
        if (vol < 0) {
            int s = q[2]; q[2] = q[3]; q[3] = s;
            m->flipped[t] = 1;
            vol = tet_volume(&m->rest[3 * q[0]], &m->rest[3 * q[1]], &m->rest[3 * q[2]], &m->rest[3 * q[3]]);
        }
        REAL L3 = m->extent * m->extent * m->extent;
        if (!(vol > 1e-12 * L3)) { orc_mesh_destroy(m); *err = ORC_E_DEGENERATE; return NULL; }
        for (int k = 0; k < 4; ++k) m->tet[4 * t + k] = q[k];
        m->V0[t] = vol;
    }
    /* edges: the six vertex pairs of every tet, as (min, max), sorted, unique */
    int* pairs;
    int np;
    if (edges_in) {
        np = n_edges_in;
        pairs = (int*)malloc(sizeof(int) * 2 * (np > 0 ? np : 1));
        for (int e = 0; e < np; ++e) {
            int a = edges_in[2 * e], b = edges_in[2 * e + 1];
            if (a < 0 || a >= V || b < 0 || b >= V || a == b) { free(pairs); orc_mesh_destroy(m); return NULL; }
            pairs[2 * e] = a < b ? a : b;
            pairs[2 * e + 1] = a < b ? b : a;
        }
    } else {
        np = 6 * T;
        pairs = (int*)malloc(sizeof(int) * 2 * (np > 0 ? np : 1));
        static const int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {1, 2, 3, 2, 3, 3};
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < 6; ++k) {
                int a = m->tet[4 * t + PA[k]], b = m->tet[4 * t + PB[k]];
                pairs[2 * (6 * t + k)] = a < b ? a : b;
                pairs[2 * (6 * t + k) + 1] = a < b ? b : a;
            }
    }
    qsort(pairs, (size_t)np, sizeof(int) * 2, cmp_pair);
    int E = 0;
    for (int p = 0; p < np; ++p)
        if (E == 0 || cmp_pair(&pairs[2 * p], &pairs[2 * (E - 1)]) != 0) {
            pairs[2 * E] = pairs[2 * p]; pairs[2 * E + 1] = pairs[2 * p + 1]; ++E;
        }
    m->E = E;
    m->edge = (int*)malloc(sizeof(int) * 2 * (E > 0 ? E : 1));
    m->d = (REAL*)malloc(sizeof(REAL) * (E > 0 ? E : 1));
    memcpy(m->edge, pairs, sizeof(int) * 2 * E);
    free(pairs);
    for (int e = 0; e < E; ++e) {
        REAL ab[3];
        vsub(&m->rest[3 * m->edge[2 * e]], &m->rest[3 * m->edge[2 * e + 1]], ab);
        m->d[e] = vnorm(ab);
        if (!(m->d[e] > 0)) { orc_mesh_destroy(m); *err = ORC_E_DEGENERATE; return NULL; }
    }
    /* colouring (R4) */
    m->ecolor = (int*)malloc(sizeof(int) * (E > 0 ? E : 1));
    m->tcolor = (int*)malloc(sizeof(int) * (T > 0 ? T : 1));
    m->eorder = (int*)malloc(sizeof(int) * (E > 0 ? E : 1));
    m->torder = (int*)malloc(sizeof(int) * (T > 0 ? T : 1));
    int rc = color_first_fit(E, 2, m->edge, V, m->ecolor, &m->n_ecol);
    if (rc == ORC_OK) rc = color_first_fit(T, 4, m->tet, V, m->tcolor, &m->n_tcol);
    if (rc != ORC_OK) { orc_mesh_destroy(m); *err = rc; return NULL; }
    m->ecol_off = (int*)malloc(sizeof(int) * (m->n_ecol + 1));
    m->tcol_off = (int*)malloc(sizeof(int) * (m->n_tcol + 1));
    color_major(E, m->ecolor, m->n_ecol, m->eorder, m->ecol_off);
    color_major(T, m->tcolor, m->n_tcol, m->torder, m->tcol_off);
    /* top face: vertices whose z equals the largest z */
    m->top = (int*)malloc(sizeof(int) * V);
    m->n_top = 0;
    for (int i = 0; i < V; ++i)
        if (m->rest[3 * i + 2] == m->bbmax[2]) m->top[m->n_top++] = i;
    /* surface faces: each tet's four faces as sorted triples with the opposite
     * vertex; a triple that occurs once is on the surface (R13) */
    int* fr = (int*)malloc(sizeof(int) * 4 * (4 * T > 0 ? 4 * T : 1));
    static const int FA[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            int v[3] = {m->tet[4 * t + FA[k][0]], m->tet[4 * t + FA[k][1]], m->tet[4 * t + FA[k][2]]};
            for (int a = 0; a < 2; ++a)   /* sort the triple */
                for (int b = 0; b < 2 - a; ++b)
                    if (v[b] > v[b + 1]) { int tmp = v[b]; v[b] = v[b + 1]; v[b + 1] = tmp; }
            int* r = &fr[4 * (4 * t + k)];
            r[0] = v[0]; r[1] = v[1]; r[2] = v[2]; r[3] = m->tet[4 * t + FA[k][3]];
        }
    qsort(fr, (size_t)(4 * T), sizeof(int) * 4, cmp_triple);
    m->face = (int*)malloc(sizeof(int) * 3 * (4 * T > 0 ? 4 * T : 1));
    m->fopp = (int*)malloc(sizeof(int) * (4 * T > 0 ? 4 * T : 1));
    m->F = 0;
    for (int q = 0; q < 4 * T;) {
        int n = 1;
        while (q + n < 4 * T && cmp_triple(&fr[4 * q], &fr[4 * (q + n)]) == 0) ++n;
        const int* r = &fr[4 * q];
        if (n == 1 && (m->w[r[0]] > 0 || m->w[r[1]] > 0 || m->w[r[2]] > 0)) {
            m->face[3 * m->F] = r[0]; m->face[3 * m->F + 1] = r[1]; m->face[3 * m->F + 2] = r[2];
            m->fopp[m->F] = r[3];
            m->F++;
        }
        q += n;
    }
    free(fr);
    m->fcolor = (int*)malloc(sizeof(int) * (m->F > 0 ? m->F : 1));
    m->forder = (int*)malloc(sizeof(int) * (m->F > 0 ? m->F : 1));
    rc = color_first_fit(m->F, 3, m->face, V, m->fcolor, &m->n_fcol);
    if (rc != ORC_OK) { orc_mesh_destroy(m); *err = rc; return NULL; }
    m->fcol_off = (int*)malloc(sizeof(int) * (m->n_fcol + 1));
    color_major(m->F, m->fcolor, m->n_fcol, m->forder, m->fcol_off);
    rc = build_connections(m, rest, conn_radius);
    if (rc != ORC_OK) { orc_mesh_destroy(m); *err = rc; return NULL; }
    *err = ORC_OK;
    return m;
}

/* Read-only views for the test suite. which: 0 info, see below. */
void orc_mesh_faces(const orc_mesh* m, int* out /* 2 */) { out[0] = m->F; out[1] = m->n_fcol; }
void orc_mesh_conns(const orc_mesh* m, int* out /* 3 */) { out[0] = m->C; out[1] = m->n_ccol; out[2] = m->n_obj; }

void orc_mesh_info(const orc_mesh* m, int* out /* 6 */) {
    out[0] = m->V; out[1] = m->T; out[2] = m->E;
    out[3] = m->n_ecol; out[4] = m->n_tcol; out[5] = m->n_top;
}
/* which: 0 tet[4T], 1 flipped[T], 2 edge[2E], 3 ecolor[E], 4 tcolor[T],
 *        5 eorder[E], 6 torder[T], 7 ecol_off, 8 tcol_off, 9 top */
int orc_mesh_get_int(const orc_mesh* m, int which, int* out) {
    switch (which) {
    case 0: memcpy(out, m->tet, sizeof(int) * 4 * m->T); break;
    case 1: memcpy(out, m->flipped, sizeof(int) * m->T); break;
    case 2: memcpy(out, m->edge, sizeof(int) * 2 * m->E); break;
    case 3: memcpy(out, m->ecolor, sizeof(int) * m->E); break;
    case 4: memcpy(out, m->tcolor, sizeof(int) * m->T); break;
    case 5: memcpy(out, m->eorder, sizeof(int) * m->E); break;
    case 6: memcpy(out, m->torder, sizeof(int) * m->T); break;
    case 7: memcpy(out, m->ecol_off, sizeof(int) * (m->n_ecol + 1)); break;
    case 8: memcpy(out, m->tcol_off, sizeof(int) * (m->n_tcol + 1)); break;
    case 9: memcpy(out, m->top, sizeof(int) * m->n_top); break;
    case 10: memcpy(out, m->face, sizeof(int) * 3 * m->F); break;
    case 11: memcpy(out, m->fopp, sizeof(int) * m->F); break;
    case 12: memcpy(out, m->forder, sizeof(int) * m->F); break;
    case 13: memcpy(out, m->fcol_off, sizeof(int) * (m->n_fcol + 1)); break;
    case 14: memcpy(out, m->conn, sizeof(int) * 4 * m->C); break;
    case 15: memcpy(out, m->corder, sizeof(int) * m->C); break;
    case 16: memcpy(out, m->ccol_off, sizeof(int) * (m->n_ccol + 1)); break;
    case 17: memcpy(out, m->obj, sizeof(int) * m->V); break;
    default: return ORC_E_INVAL;
    }
    return ORC_OK;
}
/* which: 0 d[E], 1 V0[T], 2 bbmin[3], 3 bbmax[3], 4 extent */
int orc_mesh_get_real(const orc_mesh* m, int which, double* out) {
    switch (which) {
    case 0: for (int e = 0; e < m->E; ++e) out[e] = m->d[e]; break;
    case 1: for (int t = 0; t < m->T; ++t) out[t] = m->V0[t]; break;
    case 2: for (int k = 0; k < 3; ++k) out[k] = m->bbmin[k]; break;
    case 3: for (int k = 0; k < 3; ++k) out[k] = m->bbmax[k]; break;
    case 4: out[0] = m->extent; break;
    case 5: for (int c = 0; c < m->C; ++c) out[c] = m->cd0[c]; break;
    default: return ORC_E_INVAL;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Constraint projections (Eq. 1, Eqs. 2-3, readings R1-R3, R8).             */
/* ------------------------------------------------------------------------ */

/* Distance constraint C = |x_a - x_b| - d. Gradient wrt x_a is n = x_ab/|x_ab|,
 * wrt x_b is -n. The multiplier step dl = (-C - alpha~ lambda) / (w_a + w_b +
 * alpha~) and the corrections da = w_a dl n, db = -w_b dl n at the given
 * positions (zero, with dl = 0, for a skipped constraint, R8). Returns C. */
static REAL edge_step(const REAL* xa, const REAL* xb, REAL wa, REAL wb, REAL d, REAL alpha_t, REAL lambda,
                      REAL min_len, REAL* dl_out, REAL* da, REAL* db) {
    REAL ab[3];
    vsub(xa, xb, ab);
    REAL len = vnorm(ab);
    REAL C = len - d;
    REAL denom = wa + wb + alpha_t;
    *dl_out = 0;
    for (int k = 0; k < 3; ++k) { da[k] = 0; db[k] = 0; }
    if (len < min_len || denom == 0) return C;
    REAL n[3] = {ab[0] / len, ab[1] / len, ab[2] / len};
    REAL dl = (-C - alpha_t * lambda) / denom;
    for (int k = 0; k < 3; ++k) {
        da[k] = wa * dl * n[k];
        db[k] = -(wb * dl * n[k]);
    }
    *dl_out = dl;
    return C;
}

/* Gauss-Seidel projection of one distance constraint: the step above,
 * applied at once. Returns the constraint value before the update. */
REAL orc_project_edge(REAL* xa, REAL* xb, REAL wa, REAL wb, REAL d, REAL alpha_t,
                      REAL* lambda, REAL min_len) {
    REAL dl, da[3], db[3];
    REAL C = edge_step(xa, xb, wa, wb, d, alpha_t, *lambda, min_len, &dl, da, db);
    for (int k = 0; k < 3; ++k) {
        xa[k] += da[k];
        xb[k] += db[k];
    }
    *lambda += dl;
    return C;
}

/* Volume constraint C = (x_ba x x_ca).x_da / 6 - V0 with the gradients of R1:
 * the multiplier step dl = (-C - alpha~ lambda) / (sum_i w_i |g_i|^2 + alpha~)
 * and the corrections dx_i = w_i dl g_i at the given positions. Returns C. */
static REAL tet_step(const REAL* xa, const REAL* xb, const REAL* xc, const REAL* xd, const REAL* w4, REAL V0,
                     REAL alpha_t, REAL lambda, REAL* dl_out, REAL dx[4][3]) {
    REAL ba[3], ca[3], da[3], g[4][3];
    vsub(xb, xa, ba); vsub(xc, xa, ca); vsub(xd, xa, da);
    vcross(ca, da, g[1]);
    vcross(da, ba, g[2]);
    vcross(ba, ca, g[3]);
    for (int k = 0; k < 3; ++k) {
        g[1][k] /= 6; g[2][k] /= 6; g[3][k] /= 6;
        g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);
    }
    REAL C = tet_volume(xa, xb, xc, xd) - V0; /* C^v by its definition */
    REAL denom = alpha_t;
    for (int i = 0; i < 4; ++i) denom += w4[i] * vdot(g[i], g[i]);
    *dl_out = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) dx[i][k] = 0;
    if (denom == 0) return C;
    REAL dl = (-C - alpha_t * lambda) / denom;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) dx[i][k] = w4[i] * dl * g[i][k];
    *dl_out = dl;
    return C;
}

/* Gauss-Seidel projection of one volume constraint (the step, applied). */
REAL orc_project_tet(REAL* xa, REAL* xb, REAL* xc, REAL* xd, const REAL* w4, REAL V0,
                     REAL alpha_t, REAL* lambda) {
    REAL dl, dx[4][3];
    REAL C = tet_step(xa, xb, xc, xd, w4, V0, alpha_t, *lambda, &dl, dx);
    REAL* x[4] = {xa, xb, xc, xd};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) x[i][k] += dx[i][k];
    *lambda += dl;
    return C;
}

/* Tissue connection (R16): C = |x_v - p| - d0 with p = (x_a + x_b + x_c) / 3.
 * Gradients: n = (x_v - p)/|x_v - p| at v, -n/3 at a, b and c, so
 * sum w |g|^2 = w_v + (w_a + w_b + w_c) / 9. Multiplier step and corrections
 * as in R2 (skipped as in R8 when |x_v - p| is below min_len or the
 * denominator is zero). Returns C. */
static REAL conn_step(const REAL* xv, const REAL* xa, const REAL* xb, const REAL* xc, const REAL* w4, REAL d0,
                      REAL alpha_t, REAL lambda, REAL min_len, REAL* dl_out, REAL dx[4][3]) {
    REAL p[3], r[3];
    for (int k = 0; k < 3; ++k) p[k] = (xa[k] + xb[k] + xc[k]) / 3;
    vsub(xv, p, r);
    const REAL len = vnorm(r);
    const REAL C = len - d0;
    const REAL denom = w4[0] + (w4[1] + w4[2] + w4[3]) / 9 + alpha_t;
    *dl_out = 0;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) dx[i][k] = 0;
    if (len < min_len || denom == 0) return C;
    const REAL dl = (-C - alpha_t * lambda) / denom;
    for (int k = 0; k < 3; ++k) {
        const REAL n = r[k] / len;
        dx[0][k] = w4[0] * dl * n;
        for (int i = 1; i < 4; ++i) dx[i][k] = -(w4[i] * dl * n / 3);
    }
    *dl_out = dl;
    return C;
}

/* Gauss-Seidel projection of one tissue connection (the step, applied). */
REAL orc_project_conn(REAL* xv, REAL* xa, REAL* xb, REAL* xc, const REAL* w4, REAL d0, REAL alpha_t,
                      REAL* lambda, REAL min_len) {
    REAL dl, dx[4][3];
    REAL C = conn_step(xv, xa, xb, xc, w4, d0, alpha_t, *lambda, min_len, &dl, dx);
    REAL* x[4] = {xv, xa, xb, xc};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) x[i][k] += dx[i][k];
    *lambda += dl;
    return C;
}

/* ------------------------------------------------------------------------ */
/* Environment: parameters, state, reset and step.                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    double dt;
    int substeps, iterations;
    double gravity[3];
    double alpha_d, alpha_v;   /* compliance of distance / volume constraints */
    double radius;             /* sphere tool radius */
    double action_scale;       /* tool displacement per step for |a| = 1 */
    double margin_xy, margin_below, margin_above; /* tool box (R7) */
    double w_l, w_d, w_s, success_dist;           /* reward weights (Sec. IV) */
    int n_obs, max_steps;
    int solver;      /* 0: colour Gauss-Seidel (R4); 1: Jacobi with averaging (Sec. III-A, R10) */
    int auto_reset;  /* 1: a done env starts its next episode at its next step (R11) */
    int tool_model;  /* 0: sphere proxy (R6); 1: three-capsule grasper through a remote centre (R12, R13) */
    double rcm_height;                 /* remote centre of motion above the centre of the top face */
    double shaft_radius, clamp_length, clamp_radius, clamp_angle;  /* grasper capsules (R12) */
    double grasp_radius;               /* dragging: largest distance of a grasped vertex (R15) */
} orc_params;

typedef struct orc_env {
    const orc_mesh* m;
    int V;
    REAL* x;      /* [V][3] */
    REAL* v;      /* [V][3] */
    REAL* xprev;  /* [V][3] */
    REAL* lam_e;  /* [E] */
    REAL* lam_t;  /* [T] */
    REAL* lam_c;  /* [C] */
    REAL c[3];    /* tool centre */
    REAL lo[3], hi[3];
    REAL l_prev;
    int t;        /* steps since reset */
    uint64_t seed, env;   /* seed of the current episode's draws */
    uint64_t seed0;       /* seed given to reset (R11) */
    int episode;          /* episodes started by auto-reset since then */
    int done_prev;        /* the last step reported done */
    REAL clamp_angle;     /* grasper: current clamp opening (R12, R15) */
    int grasp_v;          /* grasped vertex, -1 if none (R15) */
    REAL grasp_d0;        /* its distance to the dragging point when grasped */
    int* obs;     /* [n_obs] vertex ids */
    int n_obs;
    int target;
    int n_contacts;
    int* contacts; /* ascending ids touched by the tool in the last substep */
} orc_env;

void orc_env_destroy(orc_env* s) {
    if (!s) return;
    free(s->x); free(s->v); free(s->xprev); free(s->lam_e); free(s->lam_t); free(s->lam_c);
    free(s->obs); free(s->contacts); free(s);
}

orc_env* orc_env_create(const orc_mesh* m) {
    orc_env* s = (orc_env*)calloc(1, sizeof(orc_env));
    s->m = m; s->V = m->V;
    s->x = (REAL*)calloc(3 * m->V, sizeof(REAL));
    s->v = (REAL*)calloc(3 * m->V, sizeof(REAL));
    s->xprev = (REAL*)calloc(3 * m->V, sizeof(REAL));
    s->lam_e = (REAL*)calloc(m->E > 0 ? m->E : 1, sizeof(REAL));
    s->lam_t = (REAL*)calloc(m->T > 0 ? m->T : 1, sizeof(REAL));
    s->lam_c = (REAL*)calloc(m->C > 0 ? m->C : 1, sizeof(REAL));
    s->obs = (int*)calloc(m->V, sizeof(int));
    s->contacts = (int*)calloc(m->V, sizeof(int));
    return s;
}

static REAL dist3(const REAL* a, const REAL* b) {
    REAL d[3];
    vsub(a, b, d);
    return vnorm(d);
}

/* Episode reset (Sec. III-B): rest positions, zero velocity, tool at its
 * start above the centre of the top face, fresh observation sample and
 * target vertex drawn from (seed, env). */
static int reset_state(orc_env* s, const orc_params* p, uint64_t seed, uint64_t env) {
    const orc_mesh* m = s->m;
    if (p->n_obs < 0 || p->n_obs > m->n_top || m->n_top == 0) return ORC_E_INVAL;
    for (int i = 0; i < 3 * m->V; ++i) { s->x[i] = m->rest[i]; s->v[i] = 0; }
    for (int k = 0; k < 2; ++k) {
        s->c[k] = (m->bbmin[k] + m->bbmax[k]) / 2;
        s->lo[k] = m->bbmin[k] - (REAL)p->margin_xy;
        s->hi[k] = m->bbmax[k] + (REAL)p->margin_xy;
    }
    /* the tool touches the top face: the sphere's lowest point, or the clamp tips (R12) */
    s->c[2] = m->bbmax[2] + (p->tool_model == 1 ? (REAL)(p->clamp_length * cos(p->clamp_angle) + p->clamp_radius)
                                                : (REAL)p->radius);
    s->lo[2] = m->bbmax[2] - (REAL)p->margin_below;
    s->hi[2] = m->bbmax[2] + (REAL)p->margin_above;
    s->t = 0; s->seed = seed; s->env = env;
    s->clamp_angle = (REAL)p->clamp_angle;
    s->grasp_v = -1;
    s->grasp_d0 = 0;
    s->n_obs = p->n_obs;
    int* idx = (int*)malloc(sizeof(int) * (p->n_obs > 0 ? p->n_obs : 1));
    orc_sample_indices(seed, env, m->n_top, p->n_obs, idx);
    for (int k = 0; k < p->n_obs; ++k) s->obs[k] = m->top[idx[k]];
    free(idx);
    s->target = m->top[orc_target_index(seed, env, m->n_top)];
    s->l_prev = dist3(s->c, &s->x[3 * s->target]);
    s->n_contacts = 0;
    return ORC_OK;
}

int orc_env_reset(orc_env* s, const orc_params* p, uint64_t seed, uint64_t env) {
    s->seed0 = seed;
    s->episode = 0;
    s->done_prev = 0;
    return reset_state(s, p, seed, env);
}

/* Grasper clamp opening for the next steps (radians). */
void orc_env_set_clamp(orc_env* s, double angle) { s->clamp_angle = (REAL)angle; }

/* Seed of episode k >= 1 started by auto-reset (R11). */
uint64_t orc_episode_seed(uint64_t seed0, int k) { return orc_sm64(seed0, (1ULL << 40) + (uint64_t)k); }

/* Tool-tissue collision against the sphere proxy (Sec. III-A "Collisions",
 * readings R5, R6). Records contacts when `record` is set. */
static void collide_sphere(orc_env* s, REAL r, int record) {
    const orc_mesh* m = s->m;
    if (record) s->n_contacts = 0;
    for (int i = 0; i < m->V; ++i) {
        if (m->w[i] == 0) continue;
        REAL* x = &s->x[3 * i];
        REAL d[3];
        vsub(x, s->c, d);
        REAL len = vnorm(d);
        if (len < r) {
            if (len > 0) {
                REAL n[3] = {d[0] / len, d[1] / len, d[2] / len};
                for (int k = 0; k < 3; ++k) x[k] = s->c[k] + r * n[k];
            } else {
                x[0] = s->c[0]; x[1] = s->c[1]; x[2] = s->c[2] + r;
            }
            if (record) s->contacts[s->n_contacts++] = i;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Grasper tool (Sec. III-A "Surgical tool model" and "Collisions"; R12-R14). */
/* ------------------------------------------------------------------------ */

/* Closest point of triangle (a, b, c) to point x with its barycentric
 * coordinates w[3] (R14): the Voronoi-region case analysis of Ericson,
 * Real-Time Collision Detection (2005), Sec. 5.1.5. */
static void closest_on_triangle(const REAL* x, const REAL* a, const REAL* b, const REAL* c, REAL* out, REAL* w) {
    REAL ab[3], ac[3], ax[3], bx[3], cx[3];
    vsub(b, a, ab); vsub(c, a, ac); vsub(x, a, ax); vsub(x, b, bx); vsub(x, c, cx);
    const REAL d1 = vdot(ab, ax), d2 = vdot(ac, ax);
    const REAL d3 = vdot(ab, bx), d4 = vdot(ac, bx);
    const REAL d5 = vdot(ab, cx), d6 = vdot(ac, cx);
    const REAL vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
    if (d1 <= 0 && d2 <= 0) { w[0] = 1; w[1] = 0; w[2] = 0; }                       /* vertex a */
    else if (d3 >= 0 && d4 <= d3) { w[0] = 0; w[1] = 1; w[2] = 0; }                 /* vertex b */
    else if (vc <= 0 && d1 >= 0 && d3 <= 0) {                                       /* edge ab */
        const REAL t = d1 / (d1 - d3); w[0] = 1 - t; w[1] = t; w[2] = 0;
    } else if (d6 >= 0 && d5 <= d6) { w[0] = 0; w[1] = 0; w[2] = 1; }               /* vertex c */
    else if (vb <= 0 && d2 >= 0 && d6 <= 0) {                                       /* edge ac */
        const REAL t = d2 / (d2 - d6); w[0] = 1 - t; w[1] = 0; w[2] = t;
    } else if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {                       /* edge bc */
        const REAL t = (d4 - d3) / ((d4 - d3) + (d5 - d6)); w[0] = 0; w[1] = 1 - t; w[2] = t;
    } else {                                                                        /* interior */
        const REAL den = va + vb + vc;
        w[1] = vb / den; w[2] = vc / den; w[0] = 1 - w[1] - w[2];
    }
    for (int k = 0; k < 3; ++k) out[k] = w[0] * a[k] + w[1] * b[k] + w[2] * c[k];
}

/* Closest points of segments p0-p1 and q0-q1: parameters s, t in [0, 1]
 * (Ericson, Sec. 5.1.9). */
static void closest_segments(const REAL* p0, const REAL* p1, const REAL* q0, const REAL* q1, REAL* s, REAL* t) {
    REAL d1[3], d2[3], r[3];
    vsub(p1, p0, d1); vsub(q1, q0, d2); vsub(p0, q0, r);
    const REAL a = vdot(d1, d1), e = vdot(d2, d2), f = vdot(d2, r);
    const REAL tiny = (REAL)1e-30;
    REAL ss, tt;
    if (a <= tiny && e <= tiny) { ss = 0; tt = 0; }
    else if (a <= tiny) { ss = 0; tt = f / e; tt = tt < 0 ? 0 : (tt > 1 ? 1 : tt); }
    else {
        const REAL c = vdot(d1, r);
        if (e <= tiny) { tt = 0; ss = -c / a; ss = ss < 0 ? 0 : (ss > 1 ? 1 : ss); }
        else {
            const REAL b = vdot(d1, d2), den = a * e - b * b;
            ss = den != 0 ? (b * f - c * e) / den : 0;
            ss = ss < 0 ? 0 : (ss > 1 ? 1 : ss);
            tt = (b * ss + f) / e;
            if (tt < 0) { tt = 0; ss = -c / a; ss = ss < 0 ? 0 : (ss > 1 ? 1 : ss); }
            else if (tt > 1) { tt = 1; ss = (b - c) / a; ss = ss < 0 ? 0 : (ss > 1 ? 1 : ss); }
        }
    }
    *s = ss; *t = tt;
}

/* Closest points of segment q0-q1 and triangle (a, b, c) (R14): p on the
 * triangle with barycentric w[3], q on the segment; returns |p - q|. The
 * pair is the segment's crossing of the triangle if there is one, else the
 * nearest of: each segment end against the triangle, each triangle edge
 * against the segment (in that order, ties keeping the earlier). */
REAL orc_closest_segment_triangle(const REAL* q0, const REAL* q1, const REAL* a, const REAL* b, const REAL* c,
                                  REAL* p, REAL* q, REAL* w) {
    REAL ab[3], ac[3], n[3], dq[3], aq[3];
    vsub(b, a, ab); vsub(c, a, ac); vcross(ab, ac, n); vsub(q1, q0, dq); vsub(a, q0, aq);
    const REAL den = vdot(n, dq);
    if (den != 0) {
        const REAL t = vdot(n, aq) / den;
        if (t >= 0 && t <= 1) {
            REAL y[3], py[3], wy[3];
            for (int k = 0; k < 3; ++k) y[k] = q0[k] + t * dq[k];
            closest_on_triangle(y, a, b, c, py, wy);
            if (wy[0] > 0 && wy[1] > 0 && wy[2] > 0) {   /* strictly inside: the segment crosses */
                for (int k = 0; k < 3; ++k) { p[k] = y[k]; q[k] = y[k]; w[k] = wy[k]; }
                return 0;
            }
        }
    }
    REAL best = -1;
    const REAL* ends[2] = {q0, q1};
    for (int e = 0; e < 2; ++e) {
        REAL pe[3], we[3];
        closest_on_triangle(ends[e], a, b, c, pe, we);
        const REAL d = dist3(pe, ends[e]);
        if (best < 0 || d < best) {
            best = d;
            for (int k = 0; k < 3; ++k) { p[k] = pe[k]; q[k] = ends[e][k]; w[k] = we[k]; }
        }
    }
    const REAL* tv[3] = {a, b, c};
    for (int e = 0; e < 3; ++e) {
        const REAL* u = tv[e];
        const REAL* v = tv[(e + 1) % 3];
        REAL s_, t_;
        closest_segments(q0, q1, u, v, &s_, &t_);
        REAL cq[3], cp[3];
        for (int k = 0; k < 3; ++k) { cq[k] = q0[k] + s_ * dq[k]; cp[k] = u[k] + t_ * (v[k] - u[k]); }
        const REAL d = dist3(cp, cq);
        if (d < best) {
            best = d;
            REAL we[3] = {0, 0, 0};
            we[e] = 1 - t_; we[(e + 1) % 3] = t_;
            for (int k = 0; k < 3; ++k) { p[k] = cp[k]; q[k] = cq[k]; w[k] = we[k]; }
        }
    }
    return best;
}

/* The grasper's three capsules at tool point c (R12): the shaft from the
 * remote centre of motion to c, and two clamps from c at angles +alpha and
 * -alpha from the shaft axis in the plane of the axis and the world x axis
 * (y if the axis is along x). seg [3][2][3], radius [3]. */
static void grasper_frame(const orc_env* s, const orc_params* p, REAL* rcm, REAL* d, REAL* u) {
    const orc_mesh* m = s->m;
    rcm[0] = (m->bbmin[0] + m->bbmax[0]) / 2;
    rcm[1] = (m->bbmin[1] + m->bbmax[1]) / 2;
    rcm[2] = m->bbmax[2] + (REAL)p->rcm_height;
    vsub(s->c, rcm, d);
    const REAL L = vnorm(d);
    if (L > 0) { d[0] /= L; d[1] /= L; d[2] /= L; }
    else { d[0] = 0; d[1] = 0; d[2] = -1; }
    u[0] = 1 - d[0] * d[0]; u[1] = -d[0] * d[1]; u[2] = -d[0] * d[2];   /* e_x minus its part along d */
    if (vnorm(u) < (REAL)1e-6) { u[0] = -d[1] * d[0]; u[1] = 1 - d[1] * d[1]; u[2] = -d[1] * d[2]; }
    const REAL lu = vnorm(u);
    u[0] /= lu; u[1] /= lu; u[2] /= lu;
}

/* The dragging point: the end of the closed clamps, clamp_length along the
 * shaft axis beyond the tool point (R15). */
static void dragging_point(const orc_env* s, const orc_params* p, REAL* out) {
    REAL rcm[3], d[3], u[3];
    grasper_frame(s, p, rcm, d, u);
    for (int k = 0; k < 3; ++k) out[k] = s->c[k] + (REAL)p->clamp_length * d[k];
}

static void grasper_capsules(const orc_env* s, const orc_params* p, REAL seg[3][2][3], REAL* radius) {
    REAL rcm[3], d[3], u[3];
    grasper_frame(s, p, rcm, d, u);
    const REAL ca = cos(s->clamp_angle), sa = sin(s->clamp_angle), lc = (REAL)p->clamp_length;
    for (int k = 0; k < 3; ++k) {
        seg[0][0][k] = rcm[k]; seg[0][1][k] = s->c[k];
        seg[1][0][k] = s->c[k]; seg[1][1][k] = s->c[k] + lc * (ca * d[k] + sa * u[k]);
        seg[2][0][k] = s->c[k]; seg[2][1][k] = s->c[k] + lc * (ca * d[k] - sa * u[k]);
    }
    radius[0] = (REAL)p->shaft_radius;
    radius[1] = radius[2] = (REAL)p->clamp_radius;
}

/* Read-only view for the test suite: the grasper's three capsules at the
 * env's current tool point and clamp opening (seg [3][2][3]: shaft, clamp +,
 * clamp -; radius [3]) and the dragging point (drag [3]). */
void orc_env_grasper(const orc_env* s, const orc_params* p, double* seg, double* radius, double* drag) {
    REAL sg[3][2][3], r[3], g[3];
    grasper_capsules(s, p, sg, r);
    dragging_point(s, p, g);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 3; ++k) seg[6 * i + 3 * j + k] = (double)sg[i][j][k];
    for (int i = 0; i < 3; ++i) radius[i] = (double)r[i];
    for (int k = 0; k < 3; ++k) drag[k] = (double)g[k];
}

/* Grasper-tissue collision (R13): surface faces colour by colour, each face
 * against the shaft, then the two clamps; a face whose closest point lies
 * inside a capsule is pushed out along the penetration direction by a PBD
 * step of stiffness 1 on its vertices weighted by the barycentric
 * coordinates. Records the vertices of pushed faces when `record` is set. */
static void collide_grasper(orc_env* s, const orc_params* p, int record) {
    const orc_mesh* m = s->m;
    REAL seg[3][2][3], rad[3];
    grasper_capsules(s, p, seg, rad);
    unsigned char* hit = record ? (unsigned char*)calloc((size_t)m->V, 1) : NULL;
    for (int qf = 0; qf < m->F; ++qf) {
        const int f = m->forder[qf];
        const int* v = &m->face[3 * f];
        for (int k = 0; k < 3; ++k) {
            REAL* x0 = &s->x[3 * v[0]];
            REAL* x1 = &s->x[3 * v[1]];
            REAL* x2 = &s->x[3 * v[2]];
            REAL pp[3], qq[3], w[3];
            const REAL dist = orc_closest_segment_triangle(seg[k][0], seg[k][1], x0, x1, x2, pp, qq, w);
            if (!(dist < rad[k])) continue;
            REAL n[3];
            if (dist > (REAL)1e-12 * m->extent) {
                for (int j = 0; j < 3; ++j) n[j] = (pp[j] - qq[j]) / dist;
            } else {
                /* The axis crosses the face: push radially, away from the axis
                 * through the face's centroid; if the centroid is on the axis
                 * too, into the tissue against the outward normal. */
                REAL g[3], ax[3], rel[3];
                for (int j = 0; j < 3; ++j) g[j] = (x0[j] + x1[j] + x2[j]) / 3;
                vsub(seg[k][1], seg[k][0], ax);
                vsub(g, seg[k][0], rel);
                const REAL la2 = vdot(ax, ax);
                const REAL tt = la2 > 0 ? vdot(rel, ax) / la2 : 0;
                for (int j = 0; j < 3; ++j) n[j] = rel[j] - tt * ax[j];
                REAL ln = vnorm(n);
                if (!(ln > (REAL)1e-12 * m->extent)) {
                    REAL e1[3], e2[3], e3[3];
                    vsub(x1, x0, e1); vsub(x2, x0, e2); vcross(e1, e2, n);
                    vsub(&s->x[3 * m->fopp[f]], x0, e3);
                    ln = vnorm(n);
                    if (!(ln > 0)) continue;
                    if (vdot(n, e3) < 0) ln = -ln;   /* n / ln points toward the tet: inward */
                }
                for (int j = 0; j < 3; ++j) n[j] /= ln;
            }
            const REAL C = dist - rad[k];
            const REAL den = m->w[v[0]] * w[0] * w[0] + m->w[v[1]] * w[1] * w[1] + m->w[v[2]] * w[2] * w[2];
            if (!(den > 0)) continue;
            const REAL sc = C / den;
            REAL* xs[3] = {x0, x1, x2};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) xs[i][j] -= m->w[v[i]] * w[i] * sc * n[j];
            if (record)
                for (int i = 0; i < 3; ++i)
                    if (m->w[v[i]] > 0 && w[i] > 0) hit[v[i]] = 1;
        }
    }
    if (record) {
        s->n_contacts = 0;
        for (int i = 0; i < m->V; ++i)
            if (hit[i]) s->contacts[s->n_contacts++] = i;
        free(hit);
    }
}

/* Grasp state at the start of a step (R15): with the clamps closed below 3
 * degrees an ungrasped tool takes the free vertex nearest to the dragging
 * point within grasp_radius (ties: the lower id) and keeps its distance;
 * opening the clamps to 3 degrees or more releases it. */
static void update_grasp(orc_env* s, const orc_params* p) {
    const orc_mesh* m = s->m;
    const REAL closed = (REAL)(3.0 * 3.14159265358979323846 / 180.0);
    if (!(s->clamp_angle < closed)) { s->grasp_v = -1; return; }
    if (s->grasp_v >= 0) return;
    REAL g[3];
    dragging_point(s, p, g);
    int best = -1;
    REAL bd = 0;
    for (int i = 0; i < m->V; ++i) {
        if (m->w[i] == 0) continue;
        const REAL d = dist3(&s->x[3 * i], g);
        if (d < (REAL)p->grasp_radius && (best < 0 || d < bd)) { best = i; bd = d; }
    }
    s->grasp_v = best;
    s->grasp_d0 = bd;
}

/* Dragging constraint (R15): distance d0 between the grasped vertex and the
 * dragging point, stiffness 1, the tool kinematic: the vertex moves by -C n. */
static void project_grasp(orc_env* s, const orc_params* p) {
    if (s->grasp_v < 0) return;
    REAL g[3], dv[3];
    dragging_point(s, p, g);
    REAL* x = &s->x[3 * s->grasp_v];
    vsub(x, g, dv);
    const REAL len = vnorm(dv);
    if (!(len > 0)) return;
    const REAL C = len - s->grasp_d0;
    for (int k = 0; k < 3; ++k) x[k] -= C * dv[k] / len;
}

/* One Jacobi iteration, the paper's own parallel scheme (Sec. III-A): every
 * distance and volume constraint takes its step at the positions the
 * iteration starts from, the corrections are summed per vertex, and each
 * vertex moves by its sum divided by n_i, the number of constraints of both
 * families that contain it (R10). Multipliers are carried as in R2. */
static void jacobi_iteration(orc_env* s, REAL at_d, REAL at_v, REAL min_len) {
    const orc_mesh* m = s->m;
    REAL* acc = (REAL*)calloc(3 * (size_t)m->V, sizeof(REAL));
    int* n = (int*)calloc((size_t)m->V, sizeof(int));
    for (int e = 0; e < m->E; ++e) { n[m->edge[2 * e]]++; n[m->edge[2 * e + 1]]++; }
    for (int t = 0; t < m->T; ++t)
        for (int k = 0; k < 4; ++k) n[m->tet[4 * t + k]]++;
    for (int e = 0; e < m->E; ++e) {
        int a = m->edge[2 * e], b = m->edge[2 * e + 1];
        REAL dl, da[3], db[3];
        edge_step(&s->x[3 * a], &s->x[3 * b], m->w[a], m->w[b], m->d[e], at_d, s->lam_e[e], min_len, &dl, da, db);
        for (int k = 0; k < 3; ++k) { acc[3 * a + k] += da[k]; acc[3 * b + k] += db[k]; }
        s->lam_e[e] += dl;
    }
    for (int t = 0; t < m->T; ++t) {
        const int* v4 = &m->tet[4 * t];
        REAL w4[4] = {m->w[v4[0]], m->w[v4[1]], m->w[v4[2]], m->w[v4[3]]};
        REAL dl, dx[4][3];
        tet_step(&s->x[3 * v4[0]], &s->x[3 * v4[1]], &s->x[3 * v4[2]], &s->x[3 * v4[3]], w4, m->V0[t], at_v,
                 s->lam_t[t], &dl, dx);
        for (int i = 0; i < 4; ++i)
            for (int k = 0; k < 3; ++k) acc[3 * v4[i] + k] += dx[i][k];
        s->lam_t[t] += dl;
    }
    for (int i = 0; i < m->V; ++i)
        if (n[i] > 0)
            for (int k = 0; k < 3; ++k) s->x[3 * i + k] += acc[3 * i + k] / (REAL)n[i];
    free(acc);
    free(n);
}

/* One substep (Algorithm 1's inner loop with readings R2, R4, R5). */
static void substep(orc_env* s, const orc_params* p, REAL h, REAL alpha_d, int record) {
    const orc_mesh* m = s->m;
    const REAL min_len = (REAL)1e-12 * m->extent;
    /* predict velocity and position */
    for (int i = 0; i < m->V; ++i) {
        for (int k = 0; k < 3; ++k) s->xprev[3 * i + k] = s->x[3 * i + k];
        if (m->w[i] == 0) continue;
        for (int k = 0; k < 3; ++k) {
            s->v[3 * i + k] += h * (REAL)p->gravity[k];
            s->x[3 * i + k] += h * s->v[3 * i + k];
        }
    }
    /* constraint iterations: distance colours, then volume colours */
    REAL at_d = alpha_d / (h * h);
    REAL at_v = (REAL)p->alpha_v / (h * h);
    for (int e = 0; e < m->E; ++e) s->lam_e[e] = 0;
    for (int t = 0; t < m->T; ++t) s->lam_t[t] = 0;
    for (int c = 0; c < m->C; ++c) s->lam_c[c] = 0;
    for (int it = 0; it < p->iterations; ++it) {
        if (p->solver == 1) {
            jacobi_iteration(s, at_d, at_v, min_len);
            continue;
        }
        for (int c = 0; c < m->n_ecol; ++c)
            for (int q = m->ecol_off[c]; q < m->ecol_off[c + 1]; ++q) {
                int e = m->eorder[q];
                int a = m->edge[2 * e], b = m->edge[2 * e + 1];
                orc_project_edge(&s->x[3 * a], &s->x[3 * b], m->w[a], m->w[b], m->d[e], at_d,
                                 &s->lam_e[e], min_len);
            }
        for (int c = 0; c < m->n_tcol; ++c)
            for (int q = m->tcol_off[c]; q < m->tcol_off[c + 1]; ++q) {
                int t = m->torder[q];
                const int* v4 = &m->tet[4 * t];
                REAL w4[4] = {m->w[v4[0]], m->w[v4[1]], m->w[v4[2]], m->w[v4[3]]};
                orc_project_tet(&s->x[3 * v4[0]], &s->x[3 * v4[1]], &s->x[3 * v4[2]], &s->x[3 * v4[3]],
                                w4, m->V0[t], at_v, &s->lam_t[t]);
            }
        /* tissue connections (R16), with the distance compliance */
        for (int c = 0; c < m->n_ccol; ++c)
            for (int q = m->ccol_off[c]; q < m->ccol_off[c + 1]; ++q) {
                const int k = m->corder[q];
                const int* v4 = &m->conn[4 * k];
                REAL w4[4] = {m->w[v4[0]], m->w[v4[1]], m->w[v4[2]], m->w[v4[3]]};
                orc_project_conn(&s->x[3 * v4[0]], &s->x[3 * v4[1]], &s->x[3 * v4[2]], &s->x[3 * v4[3]],
                                 w4, m->cd0[k], at_d, &s->lam_c[k], min_len);
            }
    }
    if (p->tool_model == 1) {
        project_grasp(s, p);
        collide_grasper(s, p, record);
    } else {
        collide_sphere(s, (REAL)p->radius, record);
    }
    /* velocity update */
    for (int i = 0; i < 3 * m->V; ++i) s->v[i] = (s->x[i] - s->xprev[i]) / h;
}

int orc_obs_dim(const orc_params* p) { return 3 + 3 * p->n_obs; }

/* One simulation step: tool update (R7), `substeps` substeps, then
 * observation, reward and termination (Sec. III-B, Sec. IV).
 * action: 3 numbers in [-1, 1], or NULL to draw them from the counter-based
 * stream of (seed, env, t). alpha_d < 0 selects p->alpha_d. */
int orc_env_step(orc_env* s, const orc_params* p, const double* action, double alpha_d,
                 double* obs, double* reward, unsigned char* done) {
    const orc_mesh* m = s->m;
    if (p->solver == 1 && m->C > 0) return ORC_E_INVAL;   /* R10 covers distance and volume constraints only */
    if (p->auto_reset && s->done_prev) {
        s->episode += 1;
        int rc = reset_state(s, p, orc_episode_seed(s->seed0, s->episode), s->env);
        if (rc) return rc;
        s->done_prev = 0;
    }
    double a[3];
    for (int k = 0; k < 3; ++k)
        a[k] = action ? action[k] : orc_action(s->seed, s->env, (uint64_t)s->t, k);
    for (int k = 0; k < 3; ++k) {
        REAL c = s->c[k] + (REAL)(p->action_scale * a[k]);
        if (c < s->lo[k]) c = s->lo[k];
        if (c > s->hi[k]) c = s->hi[k];
        s->c[k] = c;
    }
    REAL h = (REAL)(p->dt / p->substeps);
    REAL ad = (REAL)(alpha_d >= 0 ? alpha_d : p->alpha_d);
    if (p->tool_model == 1) update_grasp(s, p);
    for (int sub = 0; sub < p->substeps; ++sub) substep(s, p, h, ad, sub == p->substeps - 1);
    /* observation: tool centre, then the sampled surface vertices */
    if (obs) {
        for (int k = 0; k < 3; ++k) obs[k] = (double)s->c[k];
        for (int q = 0; q < s->n_obs; ++q)
            for (int k = 0; k < 3; ++k) obs[3 + 3 * q + k] = (double)s->x[3 * s->obs[q] + k];
    }
    REAL l = dist3(s->c, &s->x[3 * s->target]);
    int succ = l < (REAL)p->success_dist;
    REAL R = (REAL)p->w_l * l + (REAL)p->w_d * (l - s->l_prev) + (REAL)p->w_s * (REAL)succ;
    s->l_prev = l;
    s->t += 1;
    const int dn = ((p->max_steps > 0 && s->t >= p->max_steps) || succ) ? 1 : 0;
    s->done_prev = dn;
    if (reward) *reward = (double)R;
    if (done) *done = (unsigned char)dn;
    (void)m;
    return ORC_OK;
}

/* n steps in a row; obs [n][obs_dim], reward [n], done [n] may be NULL.
 * actions [n][3] or NULL for the counter-based stream. */
int orc_env_run(orc_env* s, const orc_params* p, int n, const double* actions, double alpha_d,
                double* obs, double* reward, unsigned char* done) {
    int od = orc_obs_dim(p);
    for (int i = 0; i < n; ++i) {
        int rc = orc_env_step(s, p, actions ? &actions[3 * i] : NULL, alpha_d,
                              obs ? &obs[(size_t)i * od] : NULL, reward ? &reward[i] : NULL,
                              done ? &done[i] : NULL);
        if (rc) return rc;
    }
    return ORC_OK;
}

/* State access for the test suite (all double arrays, [V][3] / [3]). */
void orc_env_get(const orc_env* s, double* x, double* v, double* c) {
    for (int i = 0; i < 3 * s->V; ++i) {
        if (x) x[i] = (double)s->x[i];
        if (v) v[i] = (double)s->v[i];
    }
    if (c) for (int k = 0; k < 3; ++k) c[k] = (double)s->c[k];
}
void orc_env_set(orc_env* s, const double* x, const double* v, const double* c) {
    for (int i = 0; i < 3 * s->V; ++i) {
        if (x) s->x[i] = (REAL)x[i];
        if (v) s->v[i] = (REAL)v[i];
    }
    if (c) for (int k = 0; k < 3; ++k) s->c[k] = (REAL)c[k];
}
/* ints: [0] t, [1] target, [2] n_obs, [3] n_contacts, then obs ids, then contact ids */
void orc_env_get_ints(const orc_env* s, int* out) {
    out[0] = s->t; out[1] = s->target; out[2] = s->n_obs; out[3] = s->n_contacts;
    for (int q = 0; q < s->n_obs; ++q) out[4 + q] = s->obs[q];
    for (int q = 0; q < s->n_contacts; ++q) out[4 + s->n_obs + q] = s->contacts[q];
    out[4 + s->n_obs + s->n_contacts] = s->episode;
    out[5 + s->n_obs + s->n_contacts] = s->grasp_v;
}
void orc_env_get_tool_box(const orc_env* s, double* lo, double* hi) {
    for (int k = 0; k < 3; ++k) { lo[k] = (double)s->lo[k]; hi[k] = (double)s->hi[k]; }
}
int orc_real_size(void) { return (int)sizeof(REAL); }

/* ------------------------------------------------------------------------ */
/* Learned warm-start (not in the paper; a surrogate-assisted substep added  */
/* to the method). The network is a per-vertex perceptron 15 -> 64 -> ReLU -> */
/* 64 -> ReLU -> 3 whose output, de-normalised, is added to the predicted    */
/* positions before one constraint iteration; a constraint residual above    */
/* the threshold restores the prediction and runs the full solve instead.    */
/* ------------------------------------------------------------------------ */

#define ORC_NN_IN 15
#define ORC_NN_HID 64
#define ORC_NN_OUT 3

/* Network parameters (output-major weights) and the frozen normalisation. */
typedef struct {
    double W1[ORC_NN_HID][ORC_NN_IN], b1[ORC_NN_HID];
    double W2[ORC_NN_HID][ORC_NN_HID], b2[ORC_NN_HID];
    double W3[ORC_NN_OUT][ORC_NN_HID], b3[ORC_NN_OUT];
    double in_mean[ORC_NN_IN], in_std[ORC_NN_IN];
    double out_mean[ORC_NN_OUT], out_std[ORC_NN_OUT];
    int bf16;   /* round inputs, weights and hidden activations to bfloat16 */
} orc_mlp;

/* Round to the nearest bfloat16 (ties to even) through float32. */
static double bf16r(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* y = W3 relu(W2 relu(W1 f + b1) + b2) + b3 on normalised input; returns the
 * de-normalised output. */
void orc_mlp_forward(const orc_mlp* n, const double* feat, double* out) {
    double f[ORC_NN_IN], h1[ORC_NN_HID], h2[ORC_NN_HID];
    for (int k = 0; k < ORC_NN_IN; ++k) {
        f[k] = (feat[k] - n->in_mean[k]) / n->in_std[k];
        if (n->bf16) f[k] = bf16r(f[k]);
    }
    for (int o = 0; o < ORC_NN_HID; ++o) {
        double z = n->b1[o];
        for (int k = 0; k < ORC_NN_IN; ++k) z += (n->bf16 ? bf16r(n->W1[o][k]) : n->W1[o][k]) * f[k];
        h1[o] = z > 0 ? z : 0;
        if (n->bf16) h1[o] = bf16r(h1[o]);
    }
    for (int o = 0; o < ORC_NN_HID; ++o) {
        double z = n->b2[o];
        for (int k = 0; k < ORC_NN_HID; ++k) z += (n->bf16 ? bf16r(n->W2[o][k]) : n->W2[o][k]) * h1[k];
        h2[o] = z > 0 ? z : 0;
        if (n->bf16) h2[o] = bf16r(h2[o]);
    }
    for (int o = 0; o < ORC_NN_OUT; ++o) {
        double z = n->b3[o];
        for (int k = 0; k < ORC_NN_HID; ++k) z += (n->bf16 ? bf16r(n->W3[o][k]) : n->W3[o][k]) * h2[k];
        out[o] = z * n->out_std[o] + n->out_mean[o];
    }
}

/* 1-ring of every vertex: the vertices sharing an edge with it. */
static void one_ring(const orc_mesh* m, int* off, int* nbr) {
    for (int i = 0; i <= m->V; ++i) off[i] = 0;
    for (int e = 0; e < m->E; ++e) { off[m->edge[2 * e] + 1]++; off[m->edge[2 * e + 1] + 1]++; }
    for (int i = 0; i < m->V; ++i) off[i + 1] += off[i];
    int* fill = (int*)calloc((size_t)(m->V > 0 ? m->V : 1), sizeof(int));
    for (int e = 0; e < m->E; ++e) {
        int a = m->edge[2 * e], b = m->edge[2 * e + 1];
        nbr[off[a] + fill[a]++] = b;
        nbr[off[b] + fill[b]++] = a;
    }
    free(fill);
}

/* Features of every vertex from predicted positions xh and velocities vh:
 * displacement from rest, velocity, 1-ring mean position and velocity as
 * offsets from the vertex, offset from the tool centre. */
static void features(const orc_env* s, const REAL* xh, const REAL* vh, double* F) {
    const orc_mesh* m = s->m;
    int* off = (int*)malloc(sizeof(int) * (m->V + 1));
    int* nbr = (int*)malloc(sizeof(int) * (2 * m->E + 1));
    one_ring(m, off, nbr);
    for (int i = 0; i < m->V; ++i) {
        double* f = &F[(size_t)ORC_NN_IN * i];
        double mx[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
        int deg = off[i + 1] - off[i];
        for (int q = off[i]; q < off[i + 1]; ++q)
            for (int k = 0; k < 3; ++k) { mx[k] += (double)xh[3 * nbr[q] + k]; mv[k] += (double)vh[3 * nbr[q] + k]; }
        for (int k = 0; k < 3; ++k) {
            double xi = (double)xh[3 * i + k], vi = (double)vh[3 * i + k];
            f[k] = xi - (double)m->rest[3 * i + k];
            f[3 + k] = vi;
            f[6 + k] = deg ? mx[k] / deg - xi : 0.0;
            f[9 + k] = deg ? mv[k] / deg - vi : 0.0;
            f[12 + k] = xi - (double)s->c[k];
        }
    }
    free(off);
    free(nbr);
}

/* Largest relative constraint violation at the current positions:
 * |C| / d for edges, |C| / |V0| for tets; NaN if any of them is NaN (W5). */
double orc_env_residual(const orc_env* s) {
    const orc_mesh* m = s->m;
    double r = 0;
    for (int e = 0; e < m->E; ++e) {
        REAL ab[3];
        vsub(&s->x[3 * m->edge[2 * e]], &s->x[3 * m->edge[2 * e + 1]], ab);
        double c = fabs((double)(vnorm(ab) - m->d[e])) / (double)m->d[e];
        if (isnan(c)) return c;
        if (c > r) r = c;
    }
    for (int t = 0; t < m->T; ++t) {
        const int* q = &m->tet[4 * t];
        double c = fabs((double)(tet_volume(&s->x[3 * q[0]], &s->x[3 * q[1]], &s->x[3 * q[2]], &s->x[3 * q[3]]) -
                                 m->V0[t])) / fabs((double)m->V0[t]);
        if (isnan(c)) return c;
        if (c > r) r = c;
    }
    return r;
}

/* Predicted state of the next substep (no change to the env): positions and
 * velocities after the prediction of Algorithm 1. */
static void predicted(const orc_env* s, const orc_params* p, REAL h, REAL* xh, REAL* vh) {
    const orc_mesh* m = s->m;
    for (int i = 0; i < m->V; ++i)
        for (int k = 0; k < 3; ++k) {
            xh[3 * i + k] = s->x[3 * i + k];
            vh[3 * i + k] = s->v[3 * i + k];
            if (m->w[i] > 0) {
                vh[3 * i + k] += h * (REAL)p->gravity[k];
                xh[3 * i + k] += h * vh[3 * i + k];
            }
        }
}

/* Features [V][15] of the next substep's predicted state. */
void orc_env_features(const orc_env* s, const orc_params* p, double* F) {
    REAL h = (REAL)(p->dt / p->substeps);
    REAL* xh = (REAL*)malloc(sizeof(REAL) * 3 * s->V);
    REAL* vh = (REAL*)malloc(sizeof(REAL) * 3 * s->V);
    predicted(s, p, h, xh, vh);
    features(s, xh, vh, F);
    free(xh);
    free(vh);
}

/* One constraint sweep (all distance colours, then all volume colours). */
static void sweep(orc_env* s, const orc_params* p, REAL h, REAL alpha_d) {
    const orc_mesh* m = s->m;
    const REAL min_len = (REAL)1e-12 * m->extent;
    REAL at_d = alpha_d / (h * h), at_v = (REAL)p->alpha_v / (h * h);
    for (int c = 0; c < m->n_ecol; ++c)
        for (int q = m->ecol_off[c]; q < m->ecol_off[c + 1]; ++q) {
            int e = m->eorder[q], a = m->edge[2 * e], b = m->edge[2 * e + 1];
            orc_project_edge(&s->x[3 * a], &s->x[3 * b], m->w[a], m->w[b], m->d[e], at_d, &s->lam_e[e], min_len);
        }
    for (int c = 0; c < m->n_tcol; ++c)
        for (int q = m->tcol_off[c]; q < m->tcol_off[c + 1]; ++q) {
            int t = m->torder[q];
            const int* v4 = &m->tet[4 * t];
            REAL w4[4] = {m->w[v4[0]], m->w[v4[1]], m->w[v4[2]], m->w[v4[3]]};
            orc_project_tet(&s->x[3 * v4[0]], &s->x[3 * v4[1]], &s->x[3 * v4[2]], &s->x[3 * v4[3]], w4, m->V0[t],
                            at_v, &s->lam_t[t]);
        }
}

/* Surrogate-assisted step: per substep predict, add the network's correction
 * to free vertices, one constraint iteration, residual check; above
 * `threshold` the prediction is restored and `n_full` iterations run instead.
 * A threshold of +inf never falls back; any other falls back unless the
 * residual is at most the threshold (so a NaN residual falls back).
 * Then collision and velocity update as in the plain substep. `fallbacks`
 * (may be NULL) receives the number of substeps that fell back; `record_R`
 * (may be NULL) the residual each substep checked [substeps] (with `net`) or
 * the residual the full solve left (without). When `record_F`/`record_T` are
 * given (and `net` is NULL) the step is the plain full solve and records, per
 * substep, the features [substeps][V][15] and the targets [substeps][V][3] =
 * positions after the full solve minus prediction. The warm-start is defined
 * with the sphere tool and the distance and volume constraints only: meshes
 * with connections (R16) and the grasper (R12-R15) are refused. */
int orc_env_step_surrogate(orc_env* s, const orc_params* p, const double* action, double alpha_d,
                           const orc_mlp* net, double threshold, int n_full, double* obs, double* reward,
                           unsigned char* done, int* fallbacks, double* record_F, double* record_T,
                           double* record_R) {
    const orc_mesh* m = s->m;
    if (m->C > 0) return ORC_E_INVAL;   /* the warm-start network sees no connections */
    if (p->tool_model != 0) return ORC_E_INVAL;   /* nor the grasper's faces and grasp */
    double a[3];
    for (int k = 0; k < 3; ++k)
        a[k] = action ? action[k] : orc_action(s->seed, s->env, (uint64_t)s->t, k);
    for (int k = 0; k < 3; ++k) {
        REAL c = s->c[k] + (REAL)(p->action_scale * a[k]);
        if (c < s->lo[k]) c = s->lo[k];
        if (c > s->hi[k]) c = s->hi[k];
        s->c[k] = c;
    }
    REAL h = (REAL)(p->dt / p->substeps);
    REAL ad = (REAL)(alpha_d >= 0 ? alpha_d : p->alpha_d);
    REAL* xh = (REAL*)malloc(sizeof(REAL) * 3 * m->V);
    REAL* vh = (REAL*)malloc(sizeof(REAL) * 3 * m->V);
    double* F = (double*)malloc(sizeof(double) * ORC_NN_IN * m->V);
    int nfb = 0;
    for (int sub = 0; sub < p->substeps; ++sub) {
        predicted(s, p, h, xh, vh);
        for (int i = 0; i < 3 * m->V; ++i) { s->xprev[i] = s->x[i]; s->x[i] = xh[i]; s->v[i] = vh[i]; }
        for (int e = 0; e < m->E; ++e) s->lam_e[e] = 0;
        for (int t = 0; t < m->T; ++t) s->lam_t[t] = 0;
        if (net) {
            features(s, xh, vh, F);
            for (int i = 0; i < m->V; ++i) {
                if (m->w[i] == 0) continue;
                double dx[3];
                orc_mlp_forward(net, &F[(size_t)ORC_NN_IN * i], dx);
                for (int k = 0; k < 3; ++k) s->x[3 * i + k] += (REAL)dx[k];
            }
            sweep(s, p, h, ad);
            /* W5: a threshold of +inf never falls back; any other threshold
             * falls back unless the residual is at most it (NaN falls back) */
            const int decide = !(isinf(threshold) && threshold > 0);
            const double r = (decide || record_R) ? orc_env_residual(s) : 0.0;
            if (record_R) record_R[sub] = r;
            if (decide && !(r <= threshold)) {
                ++nfb;
                for (int i = 0; i < 3 * m->V; ++i) s->x[i] = xh[i];
                for (int e = 0; e < m->E; ++e) s->lam_e[e] = 0;
                for (int t = 0; t < m->T; ++t) s->lam_t[t] = 0;
                for (int it = 0; it < n_full; ++it) sweep(s, p, h, ad);
            }
        } else {
            if (record_F) features(s, xh, vh, &record_F[(size_t)sub * ORC_NN_IN * m->V]);
            for (int it = 0; it < n_full; ++it) sweep(s, p, h, ad);
            if (record_R) record_R[sub] = orc_env_residual(s);
            if (record_T)
                for (int i = 0; i < 3 * m->V; ++i)
                    record_T[(size_t)sub * 3 * m->V + i] = (double)(s->x[i] - xh[i]);
        }
        collide_sphere(s, (REAL)p->radius, sub == p->substeps - 1);
        for (int i = 0; i < 3 * m->V; ++i) s->v[i] = (s->x[i] - s->xprev[i]) / h;
    }
    free(xh);
    free(vh);
    free(F);
    if (fallbacks) *fallbacks = nfb;
    if (obs) {
        for (int k = 0; k < 3; ++k) obs[k] = (double)s->c[k];
        for (int q = 0; q < s->n_obs; ++q)
            for (int k = 0; k < 3; ++k) obs[3 + 3 * q + k] = (double)s->x[3 * s->obs[q] + k];
    }
    REAL l = dist3(s->c, &s->x[3 * s->target]);
    int succ = l < (REAL)p->success_dist;
    REAL R = (REAL)p->w_l * l + (REAL)p->w_d * (l - s->l_prev) + (REAL)p->w_s * (REAL)succ;
    s->l_prev = l;
    s->t += 1;
    if (reward) *reward = (double)R;
    if (done) *done = (unsigned char)(((p->max_steps > 0 && s->t >= p->max_steps) || succ) ? 1 : 0);
    return ORC_OK;
}
