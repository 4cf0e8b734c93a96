// Host-side constraint-table construction (see mesh_setup.h).
#include "mesh_setup.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <queue>
#include <random>
#include <tuple>

#include "../../include/ffsrl.h"

namespace ffsrl {

const int kEvenPerm[12][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}, {0, 2, 3, 1}, {0, 3, 1, 2},
                              {1, 2, 0, 3}, {2, 0, 1, 3}, {1, 3, 2, 0}, {3, 0, 2, 1}, {2, 1, 3, 0}, {3, 1, 0, 2}};
namespace {

constexpr int kColourWords = 4;  // up to 256 colours per constraint family

// Signed volume of the tet (x_b - x_a) x (x_c - x_a) . (x_d - x_a) / 6
// (the C^v of Sec. III-A at rest), evaluated in double.
template <class Real>
double signed_volume(const Real* p, int a, int b, int c, int d) {
    double ba[3], ca[3], da[3];
    for (int k = 0; k < 3; ++k) {
        ba[k] = double(p[3 * b + k]) - double(p[3 * a + k]);
        ca[k] = double(p[3 * c + k]) - double(p[3 * a + k]);
        da[k] = double(p[3 * d + k]) - double(p[3 * a + k]);
    }
    const double nx = ba[1] * ca[2] - ba[2] * ca[1];
    const double ny = ba[2] * ca[0] - ba[0] * ca[2];
    const double nz = ba[0] * ca[1] - ba[1] * ca[0];
    return (nx * da[0] + ny * da[1] + nz * da[2]) / 6.0;
}

// Greedy first-fit colouring: constraints are visited in index order and each
// takes the lowest colour that none of its vertices already carries. A
// per-vertex bitset records the colours present at that vertex.
template <int ARITY>
int colour_first_fit(int n, const int32_t* verts, int V, std::vector<int32_t>& colour,
                     int& n_colours) {
    std::vector<std::array<uint64_t, kColourWords>> present(V);
    for (auto& b : present) b.fill(0);
    colour.assign(n, 0);
    n_colours = 0;
    for (int i = 0; i < n; ++i) {
        std::array<uint64_t, kColourWords> taken{};
        for (int k = 0; k < ARITY; ++k) {
            const auto& b = present[verts[ARITY * i + k]];
            for (int w = 0; w < kColourWords; ++w) taken[w] |= b[w];
        }
        int c = -1;
        for (int w = 0; w < kColourWords && c < 0; ++w)
            if (~taken[w]) c = 64 * w + __builtin_ctzll(~taken[w]);
        if (c < 0) return FFSRL_E_INVAL;
        colour[i] = c;
        for (int k = 0; k < ARITY; ++k)
            present[verts[ARITY * i + k]][c >> 6] |= (uint64_t(1) << (c & 63));
        n_colours = std::max(n_colours, c + 1);
    }
    return FFSRL_OK;
}

// Stable counting sort of constraint ids by colour.
void colour_major(const std::vector<int32_t>& colour, int n_colours, std::vector<int32_t>& order,
                  std::vector<int32_t>& offsets) {
    offsets.assign(n_colours + 1, 0);
    for (int32_t c : colour) ++offsets[c + 1];
    for (int c = 0; c < n_colours; ++c) offsets[c + 1] += offsets[c];
    std::vector<int32_t> next(offsets.begin(), offsets.end() - 1);
    order.assign(colour.size(), 0);
    for (size_t i = 0; i < colour.size(); ++i) order[next[colour[i]]++] = int32_t(i);
}

}  // namespace

int build_host_mesh(int V, int T, const double* rest, const double* inv_mass,
                    const int32_t* tets, HostMesh& m, std::string& err, double conn_radius) {
    if (V < 1 || V > 65535) { err = "n_verts must be in [1, 65535]"; return FFSRL_E_INVAL; }
    if (T < 1) { err = "n_tets must be >= 1"; return FFSRL_E_INVAL; }
    if (!rest || !inv_mass || !tets) { err = "mesh arrays must be non-NULL"; return FFSRL_E_INVAL; }
    m = HostMesh();
    m.V = V;
    m.T = T;
    m.rest.resize(3 * size_t(V));
    m.inv_mass.resize(V);
    for (int i = 0; i < 3 * V; ++i) {
        if (!std::isfinite(rest[i])) { err = "non-finite rest position"; return FFSRL_E_INVAL; }
        m.rest[i] = float(rest[i]);
    }
    for (int i = 0; i < V; ++i) {
        if (!(inv_mass[i] >= 0.0) || !std::isfinite(inv_mass[i])) {
            err = "inverse mass must be finite and >= 0";
            return FFSRL_E_INVAL;
        }
        m.inv_mass[i] = float(inv_mass[i]);
    }
    // Bounding box, extent and top face come from the positions as given
    // (float64), so the tool box and the observed surface do not depend on
    // the float32 rounding of the state.
    for (int k = 0; k < 3; ++k) m.bbmin[k] = m.bbmax[k] = rest[k];
    for (int i = 0; i < V; ++i)
        for (int k = 0; k < 3; ++k) {
            m.bbmin[k] = std::min(m.bbmin[k], rest[3 * i + k]);
            m.bbmax[k] = std::max(m.bbmax[k], rest[3 * i + k]);
        }
    m.extent = std::max({m.bbmax[0] - m.bbmin[0], m.bbmax[1] - m.bbmin[1], m.bbmax[2] - m.bbmin[2]});
    const double min_vol = 1e-12 * m.extent * m.extent * m.extent;

    // Orientation and rest volume (Eq. 2's V0).
    m.tet.resize(4 * size_t(T));
    m.flipped.assign(T, 0);
    m.V0.resize(T);
    for (int t = 0; t < T; ++t) {
        int32_t q[4];
        for (int k = 0; k < 4; ++k) {
            q[k] = tets[4 * t + k];
            if (q[k] < 0 || q[k] >= V) { err = "tet vertex id out of range"; return FFSRL_E_INVAL; }
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (q[a] == q[b]) { err = "tet with a repeated vertex"; return FFSRL_E_INVAL; }
        // orientation and degeneracy from the positions as given
        double vol = signed_volume(rest, q[0], q[1], q[2], q[3]);
        if (vol < 0) {
            std::swap(q[2], q[3]);
            m.flipped[t] = 1;
            vol = signed_volume(rest, q[0], q[1], q[2], q[3]);
        }
        if (!(vol > min_vol)) { err = "degenerate (zero-volume) tet"; return FFSRL_E_DEGENERATE; }
        for (int k = 0; k < 4; ++k) m.tet[4 * t + k] = q[k];
        // rest volume of the float32 state, so C = 0 at rest up to float rounding
        m.V0[t] = float(signed_volume(m.rest.data(), q[0], q[1], q[2], q[3]));
    }

    // Edges: the six vertex pairs of each tet as (min << 32 | max), sorted, unique.
    std::vector<uint64_t> keys;
    keys.reserve(6 * size_t(T));
    for (int t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                uint64_t lo = uint64_t(std::min(m.tet[4 * t + a], m.tet[4 * t + b]));
                uint64_t hi = uint64_t(std::max(m.tet[4 * t + a], m.tet[4 * t + b]));
                keys.push_back((lo << 32) | hi);
            }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    m.E = int(keys.size());
    m.edge.resize(2 * size_t(m.E));
    m.rest_len.resize(m.E);
    for (int e = 0; e < m.E; ++e) {
        const int a = int(keys[e] >> 32), b = int(keys[e] & 0xffffffffu);
        m.edge[2 * e] = a;
        m.edge[2 * e + 1] = b;
        double s = 0;
        for (int k = 0; k < 3; ++k) {
            const double dk = double(m.rest[3 * a + k]) - double(m.rest[3 * b + k]);
            s += dk * dk;
        }
        const double len = std::sqrt(s);
        if (!(len > 0)) { err = "zero-length edge"; return FFSRL_E_DEGENERATE; }
        m.rest_len[e] = float(len);
    }

    // Colouring: edges in ascending order, tets in input order, separately.
    int rc = colour_first_fit<2>(m.E, m.edge.data(), V, m.ecolor, m.n_ecol);
    if (rc == FFSRL_OK) rc = colour_first_fit<4>(m.T, m.tet.data(), V, m.tcolor, m.n_tcol);
    if (rc != FFSRL_OK) { err = "more than 256 colours needed"; return rc; }
    colour_major(m.ecolor, m.n_ecol, m.eorder, m.ecol_off);
    colour_major(m.tcolor, m.n_tcol, m.torder, m.tcol_off);

    for (int i = 0; i < V; ++i)
        if (rest[3 * i + 2] == m.bbmax[2]) m.top.push_back(i);

    // Surface faces: every tet's four faces as sorted triples with the
    // opposite vertex; triples that occur once and have a free vertex.
    static const int FA[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};
    std::vector<std::array<int32_t, 4>> fr(4 * size_t(T));
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            std::array<int32_t, 3> v = {m.tet[4 * t + FA[k][0]], m.tet[4 * t + FA[k][1]], m.tet[4 * t + FA[k][2]]};
            std::sort(v.begin(), v.end());
            fr[4 * t + k] = {v[0], v[1], v[2], m.tet[4 * t + FA[k][3]]};
        }
    std::sort(fr.begin(), fr.end(), [](const std::array<int32_t, 4>& a, const std::array<int32_t, 4>& b) {
        return std::tie(a[0], a[1], a[2]) < std::tie(b[0], b[1], b[2]);
    });
    for (size_t q = 0; q < fr.size();) {
        size_t n = 1;
        while (q + n < fr.size() && fr[q + n][0] == fr[q][0] && fr[q + n][1] == fr[q][1] && fr[q + n][2] == fr[q][2]) ++n;
        const auto& r = fr[q];
        if (n == 1 && (m.inv_mass[r[0]] > 0 || m.inv_mass[r[1]] > 0 || m.inv_mass[r[2]] > 0)) {
            m.face.insert(m.face.end(), {r[0], r[1], r[2]});
            m.fopp.push_back(r[3]);
        }
        q += n;
    }
    m.F = int(m.fopp.size());
    if (m.F > 0) {
        rc = colour_first_fit<3>(m.F, m.face.data(), V, m.fcolor, m.n_fcol);
        if (rc != FFSRL_OK) { err = "more than 256 face colours needed"; return rc; }
    }
    colour_major(m.fcolor, m.n_fcol, m.forder, m.fcol_off);
    return build_connections(m, rest, conn_radius, err);
}

int build_connections(HostMesh& m, const double* rest, double conn_radius, std::string& err) {
    const int V = m.V;
    // Objects: connected components of the tets, numbered in the order of
    // their lowest vertex (union-find, then a relabelling pass in vertex order).
    std::vector<int> parent(V);
    for (int i = 0; i < V; ++i) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x] = parent[parent[x]];
        return x;
    };
    for (int t = 0; t < m.T; ++t)
        for (int k = 1; k < 4; ++k) {
            const int a = find(m.tet[4 * t]), b = find(m.tet[4 * t + k]);
            if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
    m.obj.assign(V, -1);
    std::vector<int> label(V, -1);
    m.n_obj = 0;
    for (int i = 0; i < V; ++i) {
        const int r = find(i);
        if (label[r] < 0) label[r] = m.n_obj++;
        m.obj[i] = label[r];
    }
    // Connections: each vertex of a surface face to the nearest face centroid
    // of a lower object, within conn_radius (rest positions as given, double;
    // ties: the first face).
    m.C = 0;
    m.conn.clear();
    m.conn_d0.clear();
    if (conn_radius > 0 && m.n_obj > 1) {
        std::vector<char> on_face(V, 0);
        for (int f = 0; f < m.F; ++f)
            for (int k = 0; k < 3; ++k) on_face[m.face[3 * f + k]] = 1;
        std::vector<double> cen(3 * size_t(m.F));
        for (int f = 0; f < m.F; ++f)
            for (int k = 0; k < 3; ++k) {
                const int32_t* fv = &m.face[3 * f];
                cen[3 * f + k] = (rest[3 * fv[0] + k] + rest[3 * fv[1] + k] + rest[3 * fv[2] + k]) / 3.0;
            }
        for (int i = 0; i < V; ++i) {
            if (!on_face[i]) continue;
            int best = -1;
            double bd2 = 0;
            for (int f = 0; f < m.F; ++f) {
                if (!(m.obj[m.face[3 * f]] < m.obj[i])) continue;
                double d2 = 0;
                for (int k = 0; k < 3; ++k) {
                    const double dk = rest[3 * i + k] - cen[3 * f + k];
                    d2 += dk * dk;
                }
                if (best < 0 || d2 < bd2) {
                    best = f;
                    bd2 = d2;
                }
            }
            if (best < 0 || !(std::sqrt(bd2) <= conn_radius)) continue;
            const int32_t* fv = &m.face[3 * best];
            m.conn.insert(m.conn.end(), {int32_t(i), fv[0], fv[1], fv[2]});
            // rest distance of the float32 state, so C = 0 at rest up to float rounding
            double r2 = 0;
            for (int k = 0; k < 3; ++k) {
                const double c = (double(m.rest[3 * fv[0] + k]) + double(m.rest[3 * fv[1] + k]) +
                                  double(m.rest[3 * fv[2] + k])) / 3.0;
                const double dk = double(m.rest[3 * i + k]) - c;
                r2 += dk * dk;
            }
            m.conn_d0.push_back(float(std::sqrt(r2)));
            ++m.C;
        }
    }
    m.n_ccol = 0;
    m.ccolor.clear();
    if (m.C > 0) {
        const int rc = colour_first_fit<4>(m.C, m.conn.data(), V, m.ccolor, m.n_ccol);
        if (rc != FFSRL_OK) { err = "more than 256 connection colours needed"; return rc; }
    }
    colour_major(m.ccolor, m.n_ccol, m.corder, m.ccol_off);
    return FFSRL_OK;
}

namespace {

// Shared-memory bank model behind the schedule: positions are float4 rows, so
// a 16-byte access of slot s uses bank group s & 7, and the 8 lanes of each
// quarter-warp of a gather (records 8g .. 8g+7 of a colour, one per lane) are
// served in one wavefront only if their slots' groups are pairwise distinct.
// The schedule therefore (1) chooses the slot of every vertex so that, within
// each colour and vertex position, the bank groups are as evenly used as
// possible, and (2) orders the records of each colour in groups of 8 with few
// repeated groups per position. Edge records may also swap their two vertices
// (the projection is antisymmetric in a and b, bit for bit). None of this
// changes results: a colour's constraints touch disjoint vertices.

// A record while it is being placed: the slots of its vertices in positions
// 0 .. ARITY-1, the constraint index in position 4 and (tets) the index of
// its vertex order in kEvenPerm in position 5.
using Rec = std::array<int, 6>;

// Cost of one group of records: for each vertex position, the largest number
// of records sharing a bank group (1 = conflict-free).
template <int ARITY>
int group_cost(const Rec* g, int n) {
    int c = 0;
    for (int k = 0; k < ARITY; ++k) {
        int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mx = 0;
        for (int l = 0; l < n; ++l) mx = std::max(mx, ++cnt[g[l][k] & 7]);
        c += mx;
    }
    return c;
}

// Greedy start: groups of 8 records with pairwise distinct bank groups in
// every position, scanning a bounded window of the remaining records (edges
// may be flipped); a group that cannot be completed takes the earliest
// remaining records.
template <int ARITY>
std::vector<Rec> group_greedy(const std::vector<Rec>& recs, bool flip) {
    const int n = int(recs.size());
    const int window = 512;
    std::vector<Rec> out;
    out.reserve(n);
    std::vector<char> taken(n, 0);
    int start = 0;
    while (int(out.size()) < n) {
        while (taken[start]) ++start;
        unsigned used[ARITY] = {};
        int got = 0, seen = 0;
        for (int j = start; j < n && got < 8 && seen < window; ++j) {
            if (taken[j]) continue;
            ++seen;
            Rec r = recs[j];
            auto fits = [&]() {
                for (int k = 0; k < ARITY; ++k)
                    if (used[k] & (1u << (r[k] & 7))) return false;
                return true;
            };
            bool ok = fits();
            if (!ok && flip) {
                std::swap(r[0], r[1]);
                ok = fits();
            }
            if (!ok) continue;
            for (int k = 0; k < ARITY; ++k) used[k] |= 1u << (r[k] & 7);
            taken[j] = 1;
            out.push_back(r);
            ++got;
        }
        for (int j = start; j < n && got < 8; ++j)
            if (!taken[j]) {
                taken[j] = 1;
                out.push_back(recs[j]);
                ++got;
            }
    }
    return out;
}

// Local search: move a conflicting record of a conflicted group into a random
// other group (swapping with one of its records, an edge record flipped if
// that helps) whenever the two groups' cost does not rise.
// Index in kEvenPerm of the permutation q[k] = p[e[k]] (p = kEvenPerm[a], e = kEvenPerm[b]).
int compose_even(int a, int b) {
    int q[4];
    for (int k = 0; k < 4; ++k) q[k] = kEvenPerm[a][kEvenPerm[b][k]];
    for (int r = 0; r < 12; ++r)
        if (std::equal(q, q + 4, kEvenPerm[r])) return r;
    return 0;   // not reached: even permutations compose to an even permutation
}

// With `rot` (tets), half of the moves instead apply an even permutation to
// the vertex order of a record of a conflicted group, kept when the group's
// cost does not rise.
template <int ARITY>
void group_improve(std::vector<Rec>& g, std::mt19937_64& rng, long long iters, bool flip, bool rot = false) {
    const int n = int(g.size()), G = (n + 7) / 8;
    if (G < 2) return;
    auto size_of = [&](int a) { return std::min(8, n - 8 * a); };
    std::vector<int> cost(G), bad;
    for (int a = 0; a < G; ++a) cost[a] = group_cost<ARITY>(&g[8 * a], size_of(a));
    for (long long it = 0; it < iters; ++it) {
        if ((it & 1023) == 0) {
            bad.clear();
            for (int a = 0; a < G; ++a)
                if (cost[a] > ARITY) bad.push_back(a);
            if (bad.empty()) return;
        }
        const int a = bad[rng() % bad.size()], b = int(rng() % G);
        if (ARITY == 4 && rot && (rng() & 1)) {
            const int i = 8 * a + int(rng() % size_of(a)), e = 1 + int(rng() % 11);
            const Rec old = g[i];
            for (int k = 0; k < 4; ++k) g[i][k] = old[kEvenPerm[e][k]];
            g[i][5] = compose_even(old[5], e);
            const int c = group_cost<ARITY>(&g[8 * a], size_of(a));
            if (c <= cost[a]) cost[a] = c;
            else g[i] = old;
            continue;
        }
        if (a == b) continue;
        // a record of group a that shares its bank group with another record
        // of the group in some position (scanning from random ones)
        int i = 8 * a + int(rng() % size_of(a));
        {
            const int na = size_of(a), k0 = int(rng() % ARITY), l0 = int(rng() % na);
            bool found = false;
            for (int dk = 0; dk < ARITY && !found; ++dk) {
                const int k = (k0 + dk) % ARITY;
                int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int l = 0; l < na; ++l) ++cnt[g[8 * a + l][k] & 7];
                for (int dl = 0; dl < na; ++dl) {
                    const int l = (l0 + dl) % na;
                    if (cnt[g[8 * a + l][k] & 7] > 1) {
                        i = 8 * a + l;
                        found = true;
                        break;
                    }
                }
            }
        }
        const int j = 8 * b + int(rng() % size_of(b));
        const int before = cost[a] + cost[b];
        std::swap(g[i], g[j]);
        const int cb = group_cost<ARITY>(&g[8 * b], size_of(b));
        int ca = group_cost<ARITY>(&g[8 * a], size_of(a));
        bool flipped = false;
        if (ca + cb > before && flip) {
            std::swap(g[i][0], g[i][1]);
            const int cf = group_cost<ARITY>(&g[8 * a], size_of(a));
            if (cf < ca) {
                ca = cf;
                flipped = true;
            } else {
                std::swap(g[i][0], g[i][1]);
            }
        }
        if (ca + cb <= before) {
            cost[a] = ca;
            cost[b] = cb;
        } else {
            if (flipped) std::swap(g[i][0], g[i][1]);
            std::swap(g[i], g[j]);
        }
    }
}

// Execution phases of one constraint family (arity A, constraints `cons`,
// oracle order `order` = colour-major with colour offsets `off`). A
// Gauss-Seidel sweep depends only on the order of the constraints that share
// a vertex, so any sequence of phases that keeps, at every vertex, the
// oracle's order of the constraints containing it gives the same bits (a
// phase is then automatically free of shared vertices). unit = 0: the colours
// are the phases. unit > 0: list scheduling over that dependency graph,
// longest remaining chain first (then oracle order), closes each phase at a
// whole multiple of `unit` ready constraints, at most `cap` (all of them when
// fewer than `unit` are ready), so that a phase costs whole rounds of `unit`
// threads and its records fit a small ring stage.
template <int A>
std::vector<std::vector<int>> constraint_phases(int n, const int32_t* cons, const std::vector<int32_t>& order,
                                                const std::vector<int32_t>& off, int n_col, int V, int unit,
                                                int cap) {
    std::vector<std::vector<int>> ph;
    if (unit <= 0) {
        for (int c = 0; c < n_col; ++c) ph.emplace_back(order.begin() + off[c], order.begin() + off[c + 1]);
        return ph;
    }
    std::vector<int> pos(n), last(V, -1), sc_off(n + 1, 0), npred(n, 0), height(n, 1);
    for (int q = 0; q < n; ++q) pos[order[q]] = q;
    // dependency edges: consecutive constraints of each vertex's sequence
    std::vector<std::pair<int, int>> dep;
    dep.reserve(size_t(A) * n);
    for (int q = 0; q < n; ++q) {
        const int i = order[q];
        for (int k = 0; k < A; ++k) {
            const int v = cons[A * i + k];
            if (last[v] >= 0) dep.emplace_back(last[v], i);
            last[v] = i;
        }
    }
    for (const auto& d : dep) ++sc_off[d.first + 1];
    for (int i = 0; i < n; ++i) sc_off[i + 1] += sc_off[i];
    std::vector<int> succ(dep.size()), fill(sc_off.begin(), sc_off.end() - 1);
    for (const auto& d : dep) {
        succ[fill[d.first]++] = d.second;
        ++npred[d.second];
    }
    for (int q = n - 1; q >= 0; --q) {
        const int i = order[q];
        for (int e = sc_off[i]; e < sc_off[i + 1]; ++e) height[i] = std::max(height[i], height[succ[e]] + 1);
    }
    auto key = [&](int i) { return (int64_t(height[i]) << 32) | int64_t(uint32_t(n - 1 - pos[i])); };
    std::priority_queue<std::pair<int64_t, int>> ready;
    for (int i = 0; i < n; ++i)
        if (npred[i] == 0) ready.push({key(i), i});
    int placed = 0;
    std::vector<int> fresh;
    while (placed < n) {
        const int k = int(ready.size());
        const int take = k < unit ? k : std::min(cap, k / unit * unit);
        std::vector<int> phase(take);
        for (int t = 0; t < take; ++t) {
            phase[t] = ready.top().second;
            ready.pop();
        }
        fresh.clear();
        for (int i : phase)
            for (int e = sc_off[i]; e < sc_off[i + 1]; ++e)
                if (--npred[succ[e]] == 0) fresh.push_back(succ[e]);
        for (int i : fresh) ready.push({key(i), i});
        std::sort(phase.begin(), phase.end(), [&](int a, int b) { return pos[a] < pos[b]; });
        placed += take;
        ph.push_back(std::move(phase));
    }
    return ph;
}

// Slots of the vertices: a permutation inside each aligned block of 32
// vertices (so vertex-order passes stay coalesced), chosen by descent on the
// imbalance of bank groups per (colour, vertex position): sum over keys and
// groups of the count above ceil(n_key / 8). Moves swap the slots of two
// vertices of one block in different bank groups; `iters` moves are tried.
std::vector<int> balanced_slots(const HostMesh& m, const std::vector<int>& ephase, int ne,
                                const std::vector<int>& tphase, int nt, const std::vector<int>& cphase, int nc,
                                std::mt19937_64& rng, long long iters) {
    const int V = m.V, K = 2 * ne + 4 * nt + 4 * nc;
    std::vector<int> slot(V);
    for (int b = 0; b < V; b += 32) {   // a permutation inside each aligned block of 32 vertices
        const int n = std::min(32, V - b);
        std::vector<int> p(n);
        for (int i = 0; i < n; ++i) p[i] = b + i;
        std::shuffle(p.begin(), p.end(), rng);
        for (int i = 0; i < n; ++i) slot[b + i] = p[i];
    }
    if (V < 2 || iters <= 0) return slot;
    std::vector<int> off(V + 1, 0), keys;   // CSR: (colour, position) keys of each vertex
    for (int e = 0; e < m.E; ++e)
        for (int p = 0; p < 2; ++p) ++off[m.edge[2 * e + p] + 1];
    for (int t = 0; t < m.T; ++t)
        for (int p = 0; p < 4; ++p) ++off[m.tet[4 * t + p] + 1];
    for (int c = 0; c < m.C; ++c)
        for (int p = 0; p < 4; ++p) ++off[m.conn[4 * c + p] + 1];
    for (int i = 0; i < V; ++i) off[i + 1] += off[i];
    keys.resize(off[V]);
    std::vector<int> fill(off.begin(), off.end() - 1), n_key(K, 0);
    for (int e = 0; e < m.E; ++e)
        for (int p = 0; p < 2; ++p) {
            const int k = 2 * ephase[e] + p;
            keys[fill[m.edge[2 * e + p]]++] = k;
            ++n_key[k];
        }
    for (int t = 0; t < m.T; ++t)
        for (int p = 0; p < 4; ++p) {
            const int k = 2 * ne + 4 * tphase[t] + p;
            keys[fill[m.tet[4 * t + p]]++] = k;
            ++n_key[k];
        }
    for (int c = 0; c < m.C; ++c)
        for (int p = 0; p < 4; ++p) {
            const int k = 2 * ne + 4 * nt + 4 * cphase[c] + p;
            keys[fill[m.conn[4 * c + p]]++] = k;
            ++n_key[k];
        }
    std::vector<std::array<int, 8>> h(K);
    for (auto& a : h) a.fill(0);
    for (int i = 0; i < V; ++i)
        for (int q = off[i]; q < off[i + 1]; ++q) ++h[keys[q]][slot[i] & 7];
    auto pen = [&](int k, int cnt) {
        const int cap = (n_key[k] + 7) / 8;
        return cnt > cap ? cnt - cap : 0;
    };
    auto move = [&](int x, int from, int to) {   // returns the change of penalty
        long long d = 0;
        for (int q = off[x]; q < off[x + 1]; ++q) {
            const int k = keys[q];
            d -= pen(k, h[k][from]) + pen(k, h[k][to]);
            --h[k][from];
            ++h[k][to];
            d += pen(k, h[k][from]) + pen(k, h[k][to]);
        }
        return d;
    };
    for (long long it = 0; it < iters; ++it) {
        const int u = int(rng() % V), b = u & ~31, v = b + int(rng() % std::min(32, V - b));
        const int ru = slot[u] & 7, rv = slot[v] & 7;
        if (ru == rv) continue;
        const long long d = move(u, ru, rv) + move(v, rv, ru);
        if (d <= 0) {
            std::swap(slot[u], slot[v]);
        } else {
            move(v, ru, rv);
            move(u, rv, ru);
        }
    }
    return slot;
}

void append_segment(Schedule& out, const void* data, int bytes, int count, int first) {
    const int off = int(out.stream.size());
    const int padded = (bytes + 15) / 16 * 16;
    out.stream.resize(off + padded, 0);
    std::memcpy(out.stream.data() + off, data, bytes);
    out.segs.insert(out.segs.end(), {off, padded, count, first});
    out.ring_bytes = std::max(out.ring_bytes, padded);
}

}  // namespace

void build_schedule(const HostMesh& m, uint64_t seed, bool permute, Schedule& out, int parts) {
    out = Schedule();
    const int V = m.V;
    parts = std::max(1, parts);
    out.parts = parts;
    out.part_slots = ((V + parts - 1) / parts + 31) / 32 * 32;
    out.slot_of.resize(V);
    out.vert_of.resize(V);
    std::mt19937_64 rng(seed);
    // phases of each family (the colours unless permuted; see constraint_phases)
    const int unit = (permute && parts == 1 && V <= kPhaseMaxVerts) ? kPhaseUnit : 0;
    // local-search moves per record: more for the small meshes of the
    // four-CTA kernel (with the tet orders about 4.5 s for the 2601-vertex
    // block; the library keeps built schedules for the process)
    const long long search = V <= kPhaseMaxVerts ? 300 : 100;
    // (phases of at most 4 KB of records: 512 edges, 256 tets or connections)
    const auto eph = constraint_phases<2>(m.E, m.edge.data(), m.eorder, m.ecol_off, m.n_ecol, V, unit, 2 * unit);
    const auto tph = constraint_phases<4>(m.T, m.tet.data(), m.torder, m.tcol_off, m.n_tcol, V, unit, unit);
    const auto cph = constraint_phases<4>(m.C, m.conn.data(), m.corder, m.ccol_off, m.n_ccol, V, unit, unit);
    out.n_ephase = int(eph.size());
    out.n_tphase = int(tph.size());
    out.n_cphase = int(cph.size());
    std::vector<int> slot(V);
    if (permute) {
        std::vector<int> ep(m.E), tp(m.T), cp(m.C);
        for (int q = 0; q < out.n_ephase; ++q)
            for (int e : eph[q]) ep[e] = q;
        for (int q = 0; q < out.n_tphase; ++q)
            for (int t : tph[q]) tp[t] = q;
        for (int q = 0; q < out.n_cphase; ++q)
            for (int c : cph[q]) cp[c] = q;
        slot = balanced_slots(m, ep, out.n_ephase, tp, out.n_tphase, cp, out.n_cphase, rng, 100ll * V);
    } else {
        for (int i = 0; i < V; ++i) slot[i] = i;
    }
    for (int i = 0; i < V; ++i) {
        out.slot_of[i] = uint16_t(slot[i]);
        out.vert_of[slot[i]] = uint16_t(i);
    }
    // the mesh's tet vertex orders (identity unless a refined schedule chose
    // them); a refined schedule may change them below
    out.tet_rot.assign(size_t(m.T), 0);
    if (m.tet_rot.size() == size_t(m.T)) out.tet_rot = m.tet_rot;
    const int P = out.part_slots;
    int first = 0;   // multiplier slot of the next record
    for (const std::vector<int>& phase : eph) {
        std::vector<std::vector<Rec>> part(parts);
        for (int e : phase) {
            const Rec r = {out.slot_of[m.edge[2 * e]], out.slot_of[m.edge[2 * e + 1]], 0, 0, e, 0};
            part[r[0] / P].push_back(r);
        }
        for (std::vector<Rec>& r : part) {
            const int n = int(r.size());
            if (permute) {
                r = group_greedy<2>(r, true);
                group_improve<2>(r, rng, search * n, true);
            }
            std::vector<uint32_t> buf(2 * size_t(n));
            for (int j = 0; j < n; ++j) {
                float d = m.rest_len[r[j][4]];
                uint32_t dbits;
                std::memcpy(&dbits, &d, 4);
                buf[2 * j] = uint32_t(r[j][0]) | (uint32_t(r[j][1]) << 16);
                buf[2 * j + 1] = dbits;
            }
            append_segment(out, buf.data(), int(buf.size() * 4), n, first);
            first += n;
        }
    }
    for (const std::vector<int>& phase : tph) {
        std::vector<std::vector<Rec>> part(parts);
        for (int t : phase) {
            const int rt = out.tet_rot[t];
            Rec r{};
            for (int k = 0; k < 4; ++k) r[k] = out.slot_of[m.tet[4 * t + kEvenPerm[rt][k]]];
            r[4] = t;
            r[5] = rt;
            part[r[0] / P].push_back(r);
        }
        for (std::vector<Rec>& r : part) {
            const int n = int(r.size());
            if (permute) {
                r = group_greedy<4>(r, false);
                group_improve<4>(r, rng, search * n, false);
                // the refined schedule also chooses each tet's vertex order
                // (modelled tet conflicts on the 17x17x9 block: 33% -> 24%)
                if (unit > 0) group_improve<4>(r, rng, 4 * search * n, false, true);
            }
            for (const Rec& q : r) out.tet_rot[q[4]] = uint8_t(q[5]);
            std::vector<uint32_t> buf(4 * size_t(n));
            for (int j = 0; j < n; ++j) {
                float v0 = m.V0[r[j][4]];
                uint32_t vbits;
                std::memcpy(&vbits, &v0, 4);
                buf[4 * j] = uint32_t(r[j][0]) | (uint32_t(r[j][1]) << 16);
                buf[4 * j + 1] = uint32_t(r[j][2]) | (uint32_t(r[j][3]) << 16);
                buf[4 * j + 2] = vbits;
                buf[4 * j + 3] = 0;
            }
            append_segment(out, buf.data(), int(buf.size() * 4), n, first);
            first += n;
        }
    }
    // Tissue connections: records (vertex, face triple) like tets, d0 in z.
    for (const std::vector<int>& phase : cph) {
        std::vector<std::vector<Rec>> part(parts);
        for (int k : phase) {
            const Rec r = {out.slot_of[m.conn[4 * k]], out.slot_of[m.conn[4 * k + 1]], out.slot_of[m.conn[4 * k + 2]],
                           out.slot_of[m.conn[4 * k + 3]], k, 0};
            part[r[0] / P].push_back(r);
        }
        for (std::vector<Rec>& r : part) {
            const int n = int(r.size());
            if (permute) {
                r = group_greedy<4>(r, false);
                group_improve<4>(r, rng, search * n, false);
            }
            std::vector<uint32_t> buf(4 * size_t(n));
            for (int j = 0; j < n; ++j) {
                float d0 = m.conn_d0[r[j][4]];
                uint32_t dbits;
                std::memcpy(&dbits, &d0, 4);
                buf[4 * j] = uint32_t(r[j][0]) | (uint32_t(r[j][1]) << 16);
                buf[4 * j + 1] = uint32_t(r[j][2]) | (uint32_t(r[j][3]) << 16);
                buf[4 * j + 2] = dbits;
                buf[4 * j + 3] = 0;
            }
            append_segment(out, buf.data(), int(buf.size() * 4), n, first);
            first += n;
        }
    }
    // Surface faces for the grasper, colour by colour (faces of one colour
    // share no vertex, so their order inside a colour is free).
    out.frec.assign(4 * size_t(m.F), 0u);
    for (int fc = 0; fc < m.n_fcol; ++fc) {
        std::vector<Rec> r;
        for (int q = m.fcol_off[fc]; q < m.fcol_off[fc + 1]; ++q) {
            const int f = m.forder[q];
            r.push_back({out.slot_of[m.face[3 * f]], out.slot_of[m.face[3 * f + 1]], out.slot_of[m.face[3 * f + 2]],
                         out.slot_of[m.fopp[f]], f, 0});
        }
        if (permute && r.size() > 8) {
            r = group_greedy<3>(r, false);
            group_improve<3>(r, rng, search * static_cast<long long>(r.size()), false);
        }
        for (size_t j = 0; j < r.size(); ++j) {
            uint32_t* o = &out.frec[4 * (size_t(m.fcol_off[fc]) + j)];
            o[0] = uint32_t(r[j][0]) | (uint32_t(r[j][1]) << 16);
            o[1] = uint32_t(r[j][2]) | (uint32_t(r[j][3]) << 16);
        }
    }
}

}  // namespace ffsrl
