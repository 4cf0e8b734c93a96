"""Pins of the oracle's grasper tool (Sec. III-A "Surgical tool model" and
"Collisions"): three capsules (shaft through the remote centre of motion,
two clamps) collide with the surface faces of the tissue.

The closest-point routine is checked against brute force (dense sampling of
both the segment and the triangle); grasping takes the nearest free vertex
in reach (brute force), keeps it at its grasp distance from the lifted tool
and releases it when the clamps open; a pushed face moves out of the capsule
and repeated pushes converge to its surface; a tool pressed into the tissue
displaces it away from the tool; a tool far from the tissue leaves it exactly
as the sphere-tool step does; the surface faces of a grid block are counted
in closed form and coloured validly; the capsules and the dragging point
follow the closed forms of the remote-centre geometry (shaft through the
remote centre, clamps at +-alpha in the plane of the axis and world x, or
world y when the shaft lies along x).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs


def params(**over):
    return inputs.default_params(**over)


def _brute(q0, q1, a, b, c, n=60):
    s = np.linspace(0, 1, 4 * n)
    seg = q0[None, :] + s[:, None] * (q1 - q0)[None, :]
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    keep = (u + v) <= 1
    tri = a[None, :] + u[keep][:, None] * (b - a)[None, :] + v[keep][:, None] * (c - a)[None, :]
    d = np.linalg.norm(seg[:, None, :] - tri[None, :, :], axis=2)
    return d.min()


def test_closest_segment_triangle_against_brute_force():
    rng = np.random.default_rng(0)
    worst = 0.0
    for case in range(150):
        a, b, c = (rng.normal(size=3) for _ in range(3))
        q0, q1 = rng.normal(size=3) * 1.5, rng.normal(size=3) * 1.5
        if case % 5 == 0:   # segment through the triangle
            y = 0.3 * a + 0.3 * b + 0.4 * c
            q0, q1 = y - rng.normal(size=3), None
            q1 = 2 * y - q0
        d, p, q, w = oracle.closest_segment_triangle(q0, q1, a, b, c)
        bf = _brute(q0, q1, a, b, c)
        # the pair is consistent: p on the triangle with weights w, q on the segment
        assert np.all(w >= -1e-12) and abs(w.sum() - 1) < 1e-12
        assert np.allclose(p, w[0] * a + w[1] * b + w[2] * c, atol=1e-12)
        t = np.dot(q - q0, q1 - q0) / np.dot(q1 - q0, q1 - q0)
        assert -1e-12 <= t <= 1 + 1e-12 and np.allclose(q, q0 + t * (q1 - q0), atol=1e-12)
        assert abs(np.linalg.norm(p - q) - d) < 1e-12
        # no sampled pair is closer, and the sampling gets within its resolution
        assert d <= bf + 1e-12
        h = 2 * max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(q1 - q0)) / 60
        assert bf - d <= h, (case, d, bf)
        worst = max(worst, bf - d)
    assert worst > 0   # the brute force is coarser than the exact answer


def _single_face_env(tool_xyz, **over):
    """One tet with three pinned vertices on the bottom and a free apex; the
    grasper comes down from above."""
    s = inputs.CELL
    rest = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0.3 * s, 0.3 * s, s]], dtype=np.float64)
    w = np.array([0.0, 0.0, 0.0, 1.0 / inputs.MASS])
    m = oracle.Mesh(rest, w, np.array([[0, 1, 2, 3]], dtype=np.int32))
    return m, rest, w


def test_surface_faces_of_a_grid_block():
    for shape in [(3, 3, 2), (5, 4, 3), (9, 9, 5)]:
        nx, ny, nz = shape
        rest, w, tets = inputs.grid_block(*shape)
        m = oracle.Mesh(rest, w, tets)
        # two triangles per boundary cell face, minus the pinned bottom face
        cells = 2 * ((nx - 1) * (ny - 1) + (nx - 1) * (nz - 1) + (ny - 1) * (nz - 1))
        assert m.F == 2 * cells - 2 * (nx - 1) * (ny - 1)
        faces = m.faces
        assert np.all(faces[:, 0] < faces[:, 1]) and np.all(faces[:, 1] < faces[:, 2])
        on_box = [np.all(np.isclose(rest[f][:, k], rest[f][0, k])) for f in faces for k in range(3)]
        assert all(any(on_box[3 * i:3 * i + 3]) for i in range(len(faces)))   # every face lies on a box side
        # colouring: faces of one colour share no vertex
        off, order = m.fcol_off, m.forder
        for c in range(m.n_fcol):
            vs = faces[order[off[c]:off[c + 1]]].ravel()
            assert len(vs) == len(set(vs.tolist()))


def test_grasper_far_above_the_tissue_leaves_the_step_unchanged():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    outs = []
    for tool in (0, 1):
        p = params(tool_model=tool, radius=0.0, margin_below=-0.5, margin_above=0.6)   # box far above
        e = oracle.Env(m, p)
        e.reset(3)
        e.run(5, want_obs=False)
        outs.append(e.state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_grasper_pressed_into_the_tissue_pushes_it_away():
    """Tool driven down into the tissue for 12 steps against the same steps
    with the tool far away: the touched top-layer vertices are displaced away
    from the tool (down, or outward from the shaft axis), as a wrong push
    direction would not do; the contact list is ascending."""
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    top = rest[:, 2].max()
    act = np.array([0.3, -0.2, -1.0])
    runs = {}
    for tool in (1, None):
        p = params(tool_model=1) if tool else params(tool_model=1, margin_below=-0.5, margin_above=0.6)
        e = oracle.Env(m, p)
        e.reset(1)
        for _ in range(12):
            e.step(act)
        runs[tool] = e
    e, free = runs[1], runs[None]
    x, _, c = e.state()
    x0 = free.state()[0]
    assert c[2] < top + 1e-12   # the tool point reached the top face
    contacts = e.ints()["contacts"]
    assert len(contacts) > 0 and np.all(np.diff(contacts) > 0)
    moved = np.linalg.norm(x - x0, axis=1) > 1e-4
    assert moved.sum() >= 3
    rcm = np.array([0.0, 0.0, top + params()["rcm_height"]])
    axis = (c - rcm) / np.linalg.norm(c - rcm)
    score = 0.0
    for i in np.nonzero(moved)[0]:
        rel = x0[i] - rcm
        radial = rel - np.dot(rel, axis) * axis        # from the axis to the vertex
        dx = x[i] - x0[i]
        score += np.dot(dx, radial / (np.linalg.norm(radial) + 1e-12)) - min(dx[2], 0.0)
    assert score > 0


def test_pushed_face_ends_on_the_capsule_surface():
    """One tet with a free apex; the shaft (from the remote centre to the tool
    point) is placed so that exactly one face lies inside it. One collision
    pass moves that face out to the capsule surface (PBD with stiffness 1);
    the pinned vertices stay."""
    s = inputs.CELL
    rest = np.array([[0, 0, 0], [2 * s, 0, 0], [0, 2 * s, 0], [0.5 * s, 0.5 * s, s]], dtype=np.float64)
    w = np.array([0.0, 0.0, 0.0, 1.0 / inputs.MASS])
    m = oracle.Mesh(rest, w, np.array([[0, 1, 2, 3]], dtype=np.int32))
    r = 0.3 * s
    p = params(tool_model=1, gravity=(0.0, 0.0, 0.0), substeps=1, iterations=0, n_obs=1, action_scale=0.0,
               rcm_height=8 * s, shaft_radius=r, clamp_length=0.0, clamp_radius=0.0,
               margin_below=10 * s, margin_xy=10 * s)
    top = rest[:, 2].max()
    rcm = np.array([(rest[:, 0].min() + rest[:, 0].max()) / 2, (rest[:, 1].min() + rest[:, 1].max()) / 2,
                    top + p["rcm_height"]])
    faces = m.faces

    def dists(x, c):
        return [oracle.closest_segment_triangle(rcm, c, *x[f])[0] for f in faces]

    # the slanted face (1, 2, 3): the tool point just outside it, along its outward normal
    g = rest[[1, 2, 3]].mean(axis=0)
    nrm = np.cross(rest[2] - rest[1], rest[3] - rest[1])
    nrm /= np.linalg.norm(nrm)
    nrm = nrm if np.dot(nrm, g - rest[0]) > 0 else -nrm
    c0 = next(g + k * r * nrm for k in np.linspace(0.05, 1.0, 40)
              if sum(d < r for d in dists(rest, g + k * r * nrm)) == 1)
    e = oracle.Env(m, p)
    e.reset(0)
    e.set_state(c=c0)
    x0 = e.state()[0].copy()
    e.step(np.zeros(3))
    x1 = e.state()[0]
    before, after = dists(x0, c0), dists(x1, c0)
    i = int(np.argmin(before))
    assert before[i] < r and sum(d < r for d in before) == 1
    # one pass moves the face's closest point to the surface; the face then
    # turns about its pinned edge, so a neighbouring point may still be
    # slightly inside: the distance grows, and repeated passes (velocity
    # cleared, so only the pushes move the apex) converge to r
    assert after[i] > before[i] + 0.5 * (r - before[i])
    for _ in range(30):
        e.set_state(v=np.zeros_like(x0))
        e.step(np.zeros(3))
    assert dists(e.state()[0], c0)[i] == pytest.approx(r, rel=1e-3)
    assert np.array_equal(e.state()[0][:3], rest[:3])


def _vertical_tool_env(**over):
    """9x9x5 block, grasper straight above the centre (its shaft is vertical,
    so the dragging point is the tool point minus clamp_length in z)."""
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(tool_model=1, **over)
    e = oracle.Env(m, p)
    e.reset(2)
    return m, rest, w, p, e


def test_grasp_takes_the_nearest_free_vertex_within_the_radius():
    m, rest, w, p, e = _vertical_tool_env(clamp_angle=math.radians(1.0), grasp_radius=3e-3)
    c = e.state()[2].copy()
    c[2] = rest[:, 2].max() + p["clamp_length"] + 0.4e-3   # clamp end just above the top centre
    c[:2] = [0.0, 0.0]
    e.set_state(c=c)
    x0 = e.state()[0].copy()
    e.step(np.zeros(3))
    g = c - np.array([0.0, 0.0, p["clamp_length"]])
    d = np.linalg.norm(x0 - g, axis=1)
    d[w == 0] = np.inf
    expect = int(np.argmin(d)) if d.min() < p["grasp_radius"] else -1
    assert expect >= 0 and e.ints()["grasp"] == expect


def test_grasped_vertex_follows_the_lifted_tool_at_its_grasp_distance():
    m, rest, w, p, e = _vertical_tool_env(clamp_angle=math.radians(1.0), grasp_radius=3e-3,
                                          shaft_radius=0.0, clamp_radius=0.0)
    c = e.state()[2].copy()
    c[2] = rest[:, 2].max() + p["clamp_length"] + 0.5e-3
    e.set_state(c=c)
    x0 = e.state()[0].copy()
    e.step(np.zeros(3))
    v = e.ints()["grasp"]
    assert v >= 0
    d0 = np.linalg.norm(x0[v] - (c - np.array([0.0, 0.0, p["clamp_length"]])))
    z_before = e.state()[0][v, 2]
    for _ in range(5):
        e.step(np.array([0.0, 0.0, 1.0]))   # lift
        x, _, ct = e.state()
        g = ct - np.array([0.0, 0.0, p["clamp_length"]])
        assert abs(np.linalg.norm(x[v] - g) - d0) < 1e-12
        assert e.ints()["grasp"] == v
    assert e.state()[0][v, 2] > z_before + 5e-3   # the tissue is lifted with the tool
    e.set_clamp(math.radians(10.0))              # open: released at the next step
    e.step(np.zeros(3))
    assert e.ints()["grasp"] == -1


def test_no_grasp_with_open_clamps_or_nothing_in_reach():
    m, rest, w, p, e = _vertical_tool_env(grasp_radius=3e-3)   # clamps open at 10 degrees
    c = e.state()[2].copy()
    c[2] = rest[:, 2].max() + p["clamp_length"] + 0.5e-3
    e.set_state(c=c)
    e.step(np.zeros(3))
    assert e.ints()["grasp"] == -1
    m, rest, w, p, e = _vertical_tool_env(clamp_angle=math.radians(1.0), grasp_radius=1e-4)
    e.step(np.zeros(3))                           # the clamp end starts 1.25 mm above the surface
    assert e.ints()["grasp"] == -1


def _grasper_at(c, **over):
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(tool_model=1, **over)
    e = oracle.Env(m, p)
    e.reset(0)
    e.set_state(c=np.asarray(c, dtype=np.float64))
    return rest, p, e


@pytest.mark.parametrize("c,angle", [((0.0, 0.0, 0.03), 10.0), ((0.012, -0.007, 0.026), 25.0),
                                     ((-0.02, 0.015, 0.035), 3.0), ((0.004, 0.0, 0.02), 0.0)])
def test_grasper_geometry_closed_forms(c, angle):
    """Shaft from the remote centre (above the top-face centre by rcm_height)
    to the tool point; clamps of clamp_length leave the tool point at +-angle
    from the shaft axis, mirror images in the plane of the axis and world x;
    the dragging point lies clamp_length beyond the tool point on the axis."""
    rest, p, e = _grasper_at(c, clamp_angle=math.radians(angle))
    seg, rad, drag = e.grasper()
    c = np.asarray(c)
    rcm = np.array([(rest[:, 0].min() + rest[:, 0].max()) / 2, (rest[:, 1].min() + rest[:, 1].max()) / 2,
                    rest[:, 2].max() + p["rcm_height"]])
    assert np.allclose(seg[0, 0], rcm, atol=1e-15) and np.allclose(seg[0, 1], c, atol=1e-15)
    d = (c - rcm) / np.linalg.norm(c - rcm)
    x = np.array([1.0, 0.0, 0.0])
    u = x - np.dot(x, d) * d
    u /= np.linalg.norm(u)
    a = math.radians(angle)
    for k, sgn in ((1, 1.0), (2, -1.0)):
        assert np.allclose(seg[k, 0], c, atol=1e-15)
        arm = seg[k, 1] - c
        assert np.linalg.norm(arm) == pytest.approx(p["clamp_length"], rel=1e-12)
        assert np.dot(arm, d) == pytest.approx(p["clamp_length"] * math.cos(a), rel=1e-12, abs=1e-15)
        assert np.allclose(arm, p["clamp_length"] * (math.cos(a) * d + sgn * math.sin(a) * u), atol=1e-14)
    # mirror images: the sum lies on the axis, the difference along u
    s_ = (seg[1, 1] - c) + (seg[2, 1] - c)
    assert np.allclose(np.cross(s_, d), 0.0, atol=1e-15)
    assert np.allclose(np.cross(seg[1, 1] - seg[2, 1], u), 0.0, atol=1e-15)
    assert np.allclose(rad, [p["shaft_radius"], p["clamp_radius"], p["clamp_radius"]])
    assert np.allclose(drag, c + p["clamp_length"] * d, atol=1e-15)


def test_vertical_shaft_opens_the_clamps_along_x():
    rest, p, e = _grasper_at((0.0, 0.0, 0.03), clamp_angle=math.radians(20.0))
    seg, _, drag = e.grasper()
    L, a = p["clamp_length"], math.radians(20.0)
    c = np.array([0.0, 0.0, 0.03])
    assert np.allclose(seg[1, 1], c + L * np.array([math.sin(a), 0.0, -math.cos(a)]), atol=1e-15)
    assert np.allclose(seg[2, 1], c + L * np.array([-math.sin(a), 0.0, -math.cos(a)]), atol=1e-15)
    assert np.allclose(drag, c - np.array([0.0, 0.0, L]), atol=1e-15)


def test_shaft_along_x_falls_back_to_the_y_axis():
    """With the shaft parallel to world x the clamp plane cannot contain x;
    the clamps then open in the plane of the axis and world y."""
    rest, w, tets = inputs.grid_block(9, 9, 5)
    top = rest[:, 2].max()
    p_h = 8 * inputs.CELL
    c = (0.05, 0.0, top + p_h)            # level with the remote centre, along +x
    rest, p, e = _grasper_at(c, clamp_angle=math.radians(15.0))
    seg, _, _ = e.grasper()
    arm = seg[1, 1] - np.asarray(c)
    a = math.radians(15.0)
    L = p["clamp_length"]
    assert np.allclose(arm, L * np.array([math.cos(a), math.sin(a), 0.0]), atol=1e-15)
