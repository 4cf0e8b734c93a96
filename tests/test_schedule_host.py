"""The GPU schedule's phases, checked on the host (no GPU): the library's own
schedule builder (csrc/mesh_setup.cpp) is compiled with a small driver
(schedule_check.cpp) and run on grid blocks and a connected two-object scene.
For both slot orders every constraint lies in exactly one record, every phase
is vertex-disjoint, and every vertex meets its constraints in colour order,
so the GPU's phases give the bits of the colour-by-colour Gauss-Seidel sweep.
On the 17x17x9 block the refined phases cut the thread rounds of 256."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2503_18616_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe,
                    os.path.join(ROOT, "tests", "schedule_check.cpp"),
                    os.path.join(ROOT, "paper_2503_18616_gb300", "csrc", "mesh_setup.cpp")], check=True)
    return exe


def _run(exe, mesh, conn_radius=0.0):
    rest, w, tets = mesh
    text = "%d %d\n%s\n%s\n%s\n" % (len(rest), len(tets), " ".join(map(repr, rest.reshape(-1).tolist())),
                                    " ".join(map(repr, w.tolist())), " ".join(map(str, tets.reshape(-1).tolist())))
    out = subprocess.run([exe, repr(conn_radius)], input=text, capture_output=True, text=True, check=True).stdout
    rows = {}
    for line in out.splitlines():
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


def test_phases_keep_colour_order_with_connections(checker):
    rows = _run(checker, inputs.stacked_blocks(9, 9, 3, 3, gap=1e-3), conn_radius=6e-3)
    assert rows[0]["ok"] == 1 and rows[1]["ok"] == 1
    assert rows[1]["phases"][2] >= 1 and rows[0]["colours"][2] >= 1
