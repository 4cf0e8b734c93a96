"""Pins of the oracle's tissue connections (Sec. III-A: distance constraints
from the vertices of one object to the centroids of the faces of another).

One projection of a stiff connection puts the vertex exactly at its rest
distance from the moved centroid and conserves linear momentum for any
masses; a compliant one leaves the residual the XPBD closed form gives; the
connection table of a stacked scene equals a brute-force nearest-centroid
search, and its colouring is valid first-fit; a stacked scene at rest is a
fixed point; connections hold a free tissue block on its base under gravity
(without them it falls); Jacobi and the warm-start step refuse meshes with
connections.
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs


def _random_case(rng, w4):
    x4 = [rng.normal(size=3) * 0.01 for _ in range(4)]
    p = (x4[1] + x4[2] + x4[3]) / 3
    d0 = np.linalg.norm(x4[0] - p) * rng.uniform(0.3, 1.7)
    return x4, d0


@pytest.mark.parametrize("w4", [(1.0, 1.0, 1.0, 1.0), (2.0, 0.5, 1.0, 3.0), (0.0, 1.0, 2.0, 1.0),
                                (1.0, 0.0, 0.0, 0.0)])
def test_stiff_connection_is_met_after_one_projection_and_conserves_momentum(w4):
    rng = np.random.default_rng(1)
    for _ in range(40):
        x4, d0 = _random_case(rng, w4)
        y4, lam, C = oracle.project_conn(x4, w4, d0, 0.0)
        p = (y4[1] + y4[2] + y4[3]) / 3
        assert abs(np.linalg.norm(y4[0] - p) - d0) < 1e-14
        assert C == pytest.approx(np.linalg.norm(x4[0] - (x4[1] + x4[2] + x4[3]) / 3) - d0, abs=1e-15)
        # pinned vertices stay; the mass-weighted corrections cancel
        mom = np.zeros(3)
        for x, y, w in zip(x4, y4, w4):
            if w == 0:
                assert np.array_equal(x, y)
            else:
                mom += (y - x) / w
        if all(w > 0 for w in w4):
            assert np.max(np.abs(mom)) < 1e-15
        # every correction lies along the vertex-centroid direction
        n = x4[0] - (x4[1] + x4[2] + x4[3]) / 3
        for x, y in zip(x4, y4):
            assert np.linalg.norm(np.cross(y - x, n)) <= 1e-12 * np.linalg.norm(n)


def test_compliant_connection_leaves_the_xpbd_residual():
    rng = np.random.default_rng(2)
    w4 = (1.5, 1.0, 0.5, 2.0)
    wsum = w4[0] + (w4[1] + w4[2] + w4[3]) / 9
    for at in (0.1, 1.0, 10.0):
        x4, d0 = _random_case(rng, w4)
        C0 = np.linalg.norm(x4[0] - (x4[1] + x4[2] + x4[3]) / 3) - d0
        y4, lam, _ = oracle.project_conn(x4, w4, d0, at)
        C1 = np.linalg.norm(y4[0] - (y4[1] + y4[2] + y4[3]) / 3) - d0
        assert C1 == pytest.approx(C0 * at / (wsum + at), rel=1e-12, abs=1e-16)
        assert lam == pytest.approx(-C0 / (wsum + at), rel=1e-12)


def test_degenerate_connection_is_skipped():
    x4 = [np.zeros(3), np.array([1.0, 0, 0]), np.array([-1.0, 0.5, 0]), np.array([0.0, -0.5, 0])]
    y4, lam, C = oracle.project_conn(x4, (1, 1, 1, 1), 0.2, 0.0, min_len=1e-9)   # vertex on the centroid
    assert lam == 0.0 and all(np.array_equal(a, b) for a, b in zip(x4, y4))


@pytest.mark.parametrize("shape,gap,radius", [((3, 3, 2, 2), 1e-3, 5e-3), ((5, 4, 2, 3), 0.0, 4e-3),
                                              ((4, 4, 3, 2), 2e-3, 3.5e-3)])
def test_connection_table_equals_brute_force(shape, gap, radius):
    rest, w, tets = inputs.stacked_blocks(*shape, gap=gap)
    m = oracle.Mesh(rest, w, tets, conn_radius=radius)
    nb = shape[0] * shape[1] * shape[2]
    assert m.n_obj == 2 and np.array_equal(m.objects, np.r_[np.zeros(nb, int), np.ones(len(rest) - nb, int)])
    faces = m.faces
    obj = m.objects
    on_face = np.zeros(len(rest), bool)
    on_face[faces.reshape(-1)] = True
    expect, d0 = [], []
    for i in range(len(rest)):
        if not on_face[i]:
            continue
        cand = [f for f in range(len(faces)) if obj[faces[f, 0]] < obj[i]]
        if not cand:
            continue
        # centroids and squared distances rounded like the rule's double
        # arithmetic, so exact ties (gap 0 puts vertices on them) fall to the
        # first face as the rule says
        fc = faces[cand]
        cen = (rest[fc[:, 0]] + rest[fc[:, 1]] + rest[fc[:, 2]]) / 3.0
        r = rest[i] - cen
        d2 = (r[:, 0] * r[:, 0] + r[:, 1] * r[:, 1]) + r[:, 2] * r[:, 2]
        j = int(np.argmin(d2))
        if np.sqrt(d2[j]) <= radius:
            expect.append([i, *faces[cand[j]]])
            d0.append(np.sqrt(d2[j]))
    assert len(expect) > 0
    assert np.array_equal(m.conns, np.array(expect, dtype=np.int32).reshape(-1, 4))
    assert np.allclose(m.conn_d0, d0, rtol=1e-14, atol=0)
    # the colouring: vertex-disjoint inside a colour, first-fit across colours
    conns, order, off = m.conns, m.corder, m.ccol_off
    assert sorted(order.tolist()) == list(range(m.C))
    colour = np.empty(m.C, int)
    for c in range(m.n_ccol):
        members = order[off[c]:off[c + 1]]
        colour[members] = c
        verts = conns[members].reshape(-1)
        assert len(set(verts.tolist())) == len(verts)
        assert list(members) == sorted(members)
    for k in range(m.C):
        for c in range(colour[k]):
            assert any(set(conns[j]) & set(conns[k]) for j in range(k) if colour[j] == c)


def test_single_object_mesh_has_no_connections():
    m = oracle.Mesh(*inputs.grid_block(5, 5, 3), conn_radius=1.0)
    assert m.n_obj == 1 and m.C == 0


def test_stacked_scene_at_rest_is_a_fixed_point():
    mesh = inputs.stacked_blocks(5, 5, 3, 3, gap=1e-3)
    m = oracle.Mesh(*mesh, conn_radius=6e-3)
    assert m.C > 0
    p = inputs.default_params(gravity=(0.0, 0.0, 0.0), conn_radius=6e-3, n_obs=8)
    e = oracle.Env(m, p)
    e.reset(3)
    c = e.state()[2].copy()
    c[2] += 0.05                      # tool far above
    e.set_state(c=c)
    for _ in range(3):
        e.step(np.zeros(3))
    assert np.max(np.abs(e.state()[0] - mesh[0])) < 1e-12 * m.extent


def test_connections_hold_the_tissue_on_its_base():
    mesh = inputs.stacked_blocks(5, 5, 3, 3, gap=1e-3)
    nb = 5 * 5 * 3
    drops = {}
    for radius in (0.0, 6e-3):
        m = oracle.Mesh(*mesh, conn_radius=radius)
        p = inputs.default_params(conn_radius=radius, n_obs=8, iterations=4)
        e = oracle.Env(m, p)
        e.reset(3)
        c = e.state()[2].copy()
        c[2] += 0.05
        e.set_state(c=c)
        d = []
        for k in range(60):
            e.step(np.zeros(3))
            if k in (29, 59):
                d.append(float(np.mean(mesh[0][nb:, 2] - e.state()[0][nb:, 2])))
        drops[radius] = d
    assert drops[0.0][0] > 0.5 * 9.81 * 0.5 ** 2 * 0.8       # free fall for half a second
    assert drops[6e-3][1] < 5e-3                             # hangs on its base, sagging less than a cell,
    assert abs(drops[6e-3][1] - drops[6e-3][0]) < 1e-5       # at rest


def test_jacobi_and_warm_start_refuse_connections():
    mesh = inputs.stacked_blocks(3, 3, 2, 2, gap=1e-3)
    m = oracle.Mesh(*mesh, conn_radius=5e-3)
    e = oracle.Env(m, inputs.default_params(solver=1, conn_radius=5e-3, n_obs=4))
    e.reset(0)
    with pytest.raises(Exception):
        e.step(np.zeros(3))
    e2 = oracle.Env(m, inputs.default_params(conn_radius=5e-3, n_obs=4))
    e2.reset(0)
    net = oracle.Net.from_params({k: np.zeros_like(v) for k, v in oracle.mlp_init(0).items()})
    with pytest.raises(Exception):
        e2.step_surrogate(net, threshold=np.inf, n_full=10)
