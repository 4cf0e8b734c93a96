// Host check of the GPU schedule builder (mesh_setup.cpp): for both slot
// orders, every constraint appears in exactly one record, every phase is
// vertex-disjoint, and every vertex meets its constraints in colour order (the
// condition under which a Gauss-Seidel sweep over the phases gives the bits of
// the sweep over the colours). Reads a mesh from stdin: V T, then rest [V][3],
// inverse masses [V], tets [T][4]; argv[1] = connection radius.
// Prints one line per slot order: phases per family, thread rounds of 256,
// and ok 0/1. With argv[2] = "tables" it prints the constraint tables instead,
// one line per table: its name, then its integers.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "../paper_2503_18616_gb300/csrc/mesh_setup.h"

using namespace ffsrl;

int main(int argc, char** argv) {
    const double conn_radius = argc > 1 ? std::atof(argv[1]) : 0.0;
    int V = 0, T = 0;
    if (std::scanf("%d %d", &V, &T) != 2) return 2;
    std::vector<double> rest(3 * size_t(V)), w(V);
    std::vector<int32_t> tets(4 * size_t(T));
    for (double& x : rest)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (double& x : w)
        if (std::scanf("%lf", &x) != 1) return 2;
    for (int32_t& x : tets)
        if (std::scanf("%d", &x) != 1) return 2;
    HostMesh m;
    std::string err;
    if (build_host_mesh(V, T, rest.data(), w.data(), tets.data(), m, err, conn_radius)) {
        std::printf("mesh rejected: %s\n", err.c_str());
        return 1;
    }
    if (argc > 2 && std::string(argv[2]) == "tables") {
        auto put = [](const char* name, const std::vector<int32_t>& v) {
            std::printf("%s", name);
            for (int32_t x : v) std::printf(" %d", x);
            std::printf("\n");
        };
        put("tets", m.tet);
        put("flipped", m.flipped);
        put("edges", m.edge);
        put("ecolor", m.ecolor);
        put("tcolor", m.tcolor);
        put("eorder", m.eorder);
        put("torder", m.torder);
        put("ecol_off", m.ecol_off);
        put("tcol_off", m.tcol_off);
        put("top", m.top);
        put("faces", m.face);
        put("face_opposite", m.fopp);
        put("forder", m.forder);
        put("fcol_off", m.fcol_off);
        put("conns", m.conn);
        put("corder", m.corder);
        put("ccol_off", m.ccol_off);
        put("objects", m.obj);
        return 0;
    }
    // constraint lookup by sorted vertex tuple -> (family, colour)
    std::map<std::array<int, 4>, int> ecol, tcol, ccol, tidx;
    for (int e = 0; e < m.E; ++e) ecol[{m.edge[2 * e], m.edge[2 * e + 1], -1, -1}] = m.ecolor[e];
    for (int t = 0; t < m.T; ++t) {
        std::array<int, 4> k = {m.tet[4 * t], m.tet[4 * t + 1], m.tet[4 * t + 2], m.tet[4 * t + 3]};
        std::sort(k.begin(), k.end());
        tcol[k] = m.tcolor[t];
        tidx[k] = t;
    }
    for (int c = 0; c < m.C; ++c) ccol[{m.conn[4 * c], m.conn[4 * c + 1], m.conn[4 * c + 2], m.conn[4 * c + 3]}] = m.ccolor[c];
    long long rotated[2] = {0, 0};   // tets of the bank-aware schedule in their own / another order
    // modelled shared-memory wavefronts of the bank-aware schedule's tet records: per group of 8
    // consecutive records (one quarter-warp) and vertex position, the largest number of records
    // whose slots share a bank group (slot mod 8); and the conflict-free count (one per position)
    long long tet_wave = 0, tet_ideal = 0;
    for (int perm = 0; perm < 2; ++perm) {
        Schedule sc;
        build_schedule(m, 0x5EEDull + uint64_t(m.V), perm == 1, sc);
        const int n_seg = int(sc.segs.size() / 4);
        bool ok = n_seg == sc.n_ephase + sc.n_tphase + sc.n_cphase;
        long long rounds = 0, records = 0;
        std::map<std::array<int, 4>, int> seen;
        std::vector<int> last(V, -1);   // colour of the last constraint each vertex met (per family)
        for (int c = 0; c < n_seg; ++c) {
            const int32_t* sg = &sc.segs[4 * c];
            const int fam = c < sc.n_ephase ? 0 : c < sc.n_ephase + sc.n_tphase ? 1 : 2;
            if (c == sc.n_ephase || c == sc.n_ephase + sc.n_tphase) std::fill(last.begin(), last.end(), -1);
            rounds += (sg[2] + 255) / 256;
            std::vector<char> used(V, 0);
            std::vector<std::pair<std::array<int, 4>, int>> phase;
            for (int q = 0; q < sg[2]; ++q) {
                const uint32_t* r =
                    reinterpret_cast<const uint32_t*>(sc.stream.data() + sg[0] + (fam == 0 ? 8 : 16) * size_t(q));
                const int A = fam == 0 ? 2 : 4;
                std::array<int, 4> v = {sc.vert_of[r[0] & 0xffffu], sc.vert_of[r[0] >> 16], -1, -1};
                if (A == 4) {
                    v[2] = sc.vert_of[r[1] & 0xffffu];
                    v[3] = sc.vert_of[r[1] >> 16];
                }
                std::array<int, 4> key = v;
                int col = -1;
                if (fam == 0) {
                    if (key[0] > key[1]) std::swap(key[0], key[1]);
                    auto it = ecol.find(key);
                    if (it != ecol.end()) col = it->second;
                } else if (fam == 1) {
                    std::sort(key.begin(), key.end());
                    auto it = tcol.find(key);
                    if (it != tcol.end()) {
                        col = it->second;
                        // the record's vertex order: the tet's under the schedule's
                        // even permutation (same signed volume)
                        const int t = tidx[key];
                        if (sc.tet_rot.size() != size_t(m.T) || sc.tet_rot[t] >= 12) {
                            ok = false;
                        } else {
                            int inv = 0;
                            for (int a = 0; a < 4; ++a) {
                                if (v[a] != m.tet[4 * t + kEvenPerm[sc.tet_rot[t]][a]]) ok = false;
                                for (int b = a + 1; b < 4; ++b)
                                    inv += kEvenPerm[sc.tet_rot[t]][a] > kEvenPerm[sc.tet_rot[t]][b];
                            }
                            if (inv % 2) ok = false;
                            if (perm == 1) ++rotated[sc.tet_rot[t] != 0];
                        }
                    }
                } else {
                    auto it = ccol.find(key);
                    if (it != ccol.end()) col = it->second;
                }
                if (col < 0) ok = false;
                if (++seen[key] != 1) ok = false;
                for (int k = 0; k < A; ++k) {
                    if (used[v[k]]) ok = false;   // a phase shares no vertex
                    used[v[k]] = 1;
                    if (last[v[k]] >= col) ok = false;   // colour order at every vertex
                }
                phase.push_back({v, col});
                ++records;
            }
            for (const auto& pr : phase)
                for (int k = 0; k < 4; ++k)
                    if (pr.first[k] >= 0) last[pr.first[k]] = pr.second;
        }
        if (records != m.E + m.T + m.C) ok = false;
        if (perm == 1)
            for (int c = sc.n_ephase; c < sc.n_ephase + sc.n_tphase; ++c) {
                const int32_t* sg = &sc.segs[4 * c];
                for (int g = 0; 8 * g < sg[2]; ++g)
                    for (int k = 0; k < 4; ++k) {
                        int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, mx = 0;
                        for (int l = 8 * g; l < sg[2] && l < 8 * g + 8; ++l) {
                            const uint32_t* r = reinterpret_cast<const uint32_t*>(sc.stream.data() + sg[0] + 16 * size_t(l));
                            const int slot = (k & 1) ? int(r[k / 2] >> 16) : int(r[k / 2] & 0xffffu);
                            mx = std::max(mx, ++cnt[slot & 7]);
                        }
                        tet_wave += mx;
                        ++tet_ideal;
                    }
            }
        // grasper face records: colour by colour, every face of the colour
        // once (with its opposite vertex), no vertex twice in a colour
        if (sc.frec.size() != 4 * size_t(m.F)) ok = false;
        std::map<std::array<int, 3>, int> face_of;
        for (int f = 0; f < m.F; ++f) {
            std::array<int, 3> k = {m.face[3 * f], m.face[3 * f + 1], m.face[3 * f + 2]};
            std::sort(k.begin(), k.end());
            face_of[k] = f;
        }
        std::vector<int> face_seen(m.F, 0), fcol(m.F, -1);
        for (int fc = 0; fc < m.n_fcol; ++fc)
            for (int q = m.fcol_off[fc]; q < m.fcol_off[fc + 1]; ++q) fcol[m.forder[q]] = fc;
        for (int fc = 0; fc < m.n_fcol && sc.frec.size() == 4 * size_t(m.F); ++fc) {
            std::vector<char> used(V, 0);
            for (int q = m.fcol_off[fc]; q < m.fcol_off[fc + 1]; ++q) {
                const uint32_t* r = &sc.frec[4 * size_t(q)];
                std::array<int, 3> k = {sc.vert_of[r[0] & 0xffffu], sc.vert_of[r[0] >> 16], sc.vert_of[r[1] & 0xffffu]};
                for (int v : k) {
                    if (used[v]) ok = false;
                    used[v] = 1;
                }
                std::sort(k.begin(), k.end());
                auto it = face_of.find(k);
                if (it == face_of.end() || fcol[it->second] != fc || ++face_seen[it->second] != 1 ||
                    sc.vert_of[r[1] >> 16] != m.fopp[it->second])
                    ok = false;
            }
        }
        std::printf("permute %d phases %d %d %d colours %d %d %d rounds %lld ok %d\n", perm, sc.n_ephase, sc.n_tphase,
                    sc.n_cphase, m.n_ecol, m.n_tcol, m.n_ccol, rounds, int(ok));
    }
    std::printf("rotated %lld %lld\n", rotated[0], rotated[1]);
    std::printf("tetwaves %lld %lld\n", tet_wave, tet_ideal);
    return 0;
}
