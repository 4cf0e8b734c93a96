"""The library's host-side setup, checked without a GPU: its mesh and schedule
builder (csrc/mesh_setup.cpp) is compiled with a small driver
(schedule_check.cpp). The constraint tables (edges, oriented tets, colours and
colour-major orders, top face, surface faces, objects and tissue connections)
must equal the oracle's bit for bit, and the GPU schedule's phases are
checked on grid blocks and a connected two-object scene.
For both slot orders every constraint lies in exactly one record, every phase
is vertex-disjoint, and every vertex meets its constraints in colour order,
so the GPU's phases give the bits of the colour-by-colour Gauss-Seidel sweep.
On the 17x17x9 block the refined phases cut the thread rounds of 256.
Every tet record lists its tet's vertices in an even permutation of the
mesh's order (the signed volume and V0 unchanged): the one the schedule
reports, which the bank-aware schedule chooses."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-ffp-contract=off", "-o", exe,   # as the library build
                    os.path.join(ROOT, "tests", "schedule_check.cpp"),
                    os.path.join(ROOT, "paper_2503_18616_gb300", "csrc", "mesh_setup.cpp")], check=True)
    return exe


def _mesh_text(mesh):
    rest, w, tets = mesh
    return "%d %d\n%s\n%s\n%s\n" % (len(rest), len(tets), " ".join(map(repr, rest.reshape(-1).tolist())),
                                     " ".join(map(repr, w.tolist())), " ".join(map(str, tets.reshape(-1).tolist())))


def _run(exe, mesh, conn_radius=0.0):
    out = subprocess.run([exe, repr(conn_radius)], input=_mesh_text(mesh), capture_output=True, text=True,
                         check=True).stdout
    rows = {}
    for line in out.splitlines():
        r = re.match(r"rotated (\d+) (\d+)", line)
        if r:   # bank-aware schedule's tets in their own vertex order / in another even order
            rows["rotated"] = (int(r.group(1)), int(r.group(2)))
            continue
        r = re.match(r"tetwaves (\d+) (\d+)", line)
        if r:   # modelled shared-memory wavefronts of its tet records, and the conflict-free count
            rows["tetwaves"] = (int(r.group(1)), int(r.group(2)))
            continue
        m = re.match(r"permute (\d) phases (\d+) (\d+) (\d+) colours (\d+) (\d+) (\d+) rounds (\d+) ok (\d)", line)
        assert m, line
        g = [int(x) for x in m.groups()]
        rows[g[0]] = {"phases": g[1:4], "colours": g[4:7], "rounds": g[7], "ok": g[8]}
    return rows


@pytest.mark.parametrize("shape", [(3, 3, 2), (9, 9, 5), (17, 17, 9)])
def test_phases_keep_colour_order_on_grid_blocks(checker, shape):
    rows = _run(checker, inputs.grid_block(*shape))
    assert rows[0]["ok"] == 1 and rows[1]["ok"] == 1
    assert rows[0]["phases"] == rows[0]["colours"]          # colour phases without the permutation
    if shape == (17, 17, 9):
        assert rows[1]["phases"][:2] == [31, 43]              # 512-edge / 256-tet phases
        assert rows[1]["rounds"] == 98 and rows[0]["rounds"] == 130
        # the refined schedule reorders some tets' vertices (even permutations,
        # checked record by record above) to spread bank groups
        assert rows["rotated"][1] > 0
        # the bank-aware search keeps the tet records' modelled extra wavefronts
        # (quarter-warp groups whose slots share a bank group) at about a quarter
        # (33% in the mesh's own vertex orders, 24% with the chosen ones)
        waves, ideal = rows["tetwaves"]
        assert (waves - ideal) / waves < 0.26, (waves, ideal)


def test_phases_keep_colour_order_with_connections(checker):
    rows = _run(checker, inputs.stacked_blocks(9, 9, 3, 3, gap=1e-3), conn_radius=6e-3)
    assert rows[0]["ok"] == 1 and rows[1]["ok"] == 1
    assert rows[1]["phases"][2] >= 1 and rows[0]["colours"][2] >= 1


@pytest.mark.parametrize("case", ["two_tet", (3, 3, 2), (9, 9, 5), (17, 17, 9), "stacked", "stacked_touching"])
def test_host_tables_equal_the_oracle(checker, case):
    radius = 0.0
    if case == "two_tet":
        mesh = inputs.two_tet_mesh()
    elif case == "stacked":
        mesh, radius = inputs.stacked_blocks(9, 9, 3, 3, gap=1e-3), 6e-3
    elif case == "stacked_touching":    # exact centroid ties
        mesh, radius = inputs.stacked_blocks(5, 4, 2, 3, gap=0.0), 4e-3
    else:
        mesh = inputs.grid_block(*case)
    out = subprocess.run([checker, repr(radius), "tables"], input=_mesh_text(mesh), capture_output=True, text=True,
                         check=True).stdout
    lib = {}
    for line in out.splitlines():
        name, *vals = line.split()
        lib[name] = np.array([int(v) for v in vals], dtype=np.int64)
    om = oracle.Mesh(*mesh, conn_radius=radius)
    want = {"tets": om.tets, "flipped": om.flipped, "edges": om.edges, "ecolor": om.ecolor, "tcolor": om.tcolor,
            "eorder": om.eorder, "torder": om.torder, "ecol_off": om.ecol_off, "tcol_off": om.tcol_off,
            "top": om.top, "faces": om.faces, "face_opposite": om.face_opposite, "forder": om.forder,
            "fcol_off": om.fcol_off, "conns": om.conns, "corder": om.corder, "ccol_off": om.ccol_off,
            "objects": om.objects}
    for name, ref in want.items():
        assert np.array_equal(lib[name], np.asarray(ref).reshape(-1)), name
    if radius > 0:
        assert om.C > 0


@pytest.mark.parametrize("shape", [(10, 10, 5), (18, 18, 9), (21, 21, 11)])
def test_phases_on_uneven_batch_sizes(checker, shape):
    """Sizes of the uneven batch on both sides of the refinement limit (2944
    vertices): refined phases below it, the colours above it."""
    rows = _run(checker, inputs.grid_block(*shape))
    assert rows[0]["ok"] == 1 and rows[1]["ok"] == 1
    V = shape[0] * shape[1] * shape[2]
    if V > 2944:
        assert rows[1]["phases"] == rows[1]["colours"]
    assert rows[1]["rounds"] <= rows[0]["rounds"]
