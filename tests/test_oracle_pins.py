"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle (oracle/xpbd_oracle.c) against something other
than itself: a closed form, an invariant, a published test vector, or an
independent brute-force re-implementation. Sections of the FF-SRL paper
(arXiv 2503.18616) are cited where the fact comes from it.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 9.81
M = 1e-3


def params(**over):
    return inputs.default_params(**over)


# --------------------------------------------------------------------------
# Counter-based RNG (SplitMix64 test vector)
# --------------------------------------------------------------------------

def _golden_ints(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(int(line))
    return vals


def test_splitmix64_published_vector():
    seed, *expected = _golden_ints("splitmix64_seed1234567.txt")
    got = [oracle.sm64(seed, n) for n in range(len(expected))]
    assert got == expected


def test_uniform_mapping_uses_top_24_bits():
    assert oracle.uniform_pm1(0) == -1.0
    assert oracle.uniform_pm1((2**64) - 1) == 1.0 - 2.0**-23
    assert oracle.uniform_pm1(1 << 63) == 0.0
    # low 40 bits never matter
    assert oracle.uniform_pm1((5 << 40) | 0xFFFFFFFFFF) == oracle.uniform_pm1(5 << 40)


def test_action_stream_is_counter_based():
    seed, env = 77, 5
    st = oracle.stream(seed, env, 0)
    assert st == oracle.sm64(seed, 4 * env + 0)
    for t, axis in [(0, 0), (3, 2), (1000, 1)]:
        assert oracle.action(seed, env, t, axis) == oracle.uniform_pm1(oracle.sm64(st, 3 * t + axis))


def test_floyd_sampling_is_a_uniform_sorted_subset():
    n, k = 289, 64
    for env in range(20):
        s = oracle.sample_indices(11, env, n, k)
        assert len(s) == k and len(set(s.tolist())) == k
        assert np.all(np.diff(s) > 0) and s.min() >= 0 and s.max() < n
    # full draw returns everything; empty draw is empty
    assert oracle.sample_indices(3, 0, 10, 10).tolist() == list(range(10))
    assert len(oracle.sample_indices(3, 0, 10, 0)) == 0
    # inclusion frequency is k/n for every element (chi-square, 4000 draws)
    n, k, draws = 12, 4, 4000
    counts = np.zeros(n)
    for env in range(draws):
        counts[oracle.sample_indices(5, env, n, k)] += 1
    expect = draws * k / n
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 35.0  # 11 dof, p ~ 2.5e-4


# --------------------------------------------------------------------------
# Mesh tables (Sec. III-A: edges, rest distance, rest volume)
# --------------------------------------------------------------------------

def _grid_edge_count(nx, ny, nz):
    axis = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    faces = (nx - 1) * (ny - 1) * nz + (nx - 1) * ny * (nz - 1) + nx * (ny - 1) * (nz - 1)
    return axis + faces


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 2, 2), (4, 3, 2), (9, 9, 5), (17, 17, 9)])
def test_grid_tables_closed_form(shape):
    nx, ny, nz = shape
    rest, w, tets = inputs.grid_block(nx, ny, nz)
    m = oracle.Mesh(rest, w, tets)
    cells = (nx - 1) * (ny - 1) * (nz - 1)
    assert m.V == nx * ny * nz and m.T == 5 * cells
    # every cell face holds exactly one diagonal: axis edges + one per face
    assert m.E == _grid_edge_count(nx, ny, nz)
    s = inputs.CELL
    d = m.rest_len
    assert np.all(np.isclose(d, s, rtol=1e-14) | np.isclose(d, s * math.sqrt(2), rtol=1e-14))
    V0 = m.V0
    assert np.all(V0 > 0)
    assert np.isclose(V0.sum(), cells * s**3, rtol=1e-12)
    assert np.sum(np.isclose(V0, s**3 / 3, rtol=1e-12)) == cells
    assert np.sum(np.isclose(V0, s**3 / 6, rtol=1e-12)) == 4 * cells
    # oriented tets: flipped ones are the input with vertices 2, 3 swapped
    ot, fl = m.tets, m.flipped
    for t in range(m.T):
        exp = tets[t].copy()
        if fl[t]:
            exp[[2, 3]] = exp[[3, 2]]
        assert ot[t].tolist() == exp.tolist()
    # edges are unique, (min,max), ascending, and are exactly the tet edges
    e = m.edges
    assert np.all(e[:, 0] < e[:, 1])
    keys = e[:, 0].astype(np.int64) * m.V + e[:, 1]
    assert np.all(np.diff(keys) > 0)
    ref = sorted({tuple(sorted((int(t[a]), int(t[b])))) for t in tets
                  for a, b in itertools.combinations(range(4), 2)})
    assert [tuple(x) for x in e.tolist()] == ref
    top = m.top
    assert len(top) == nx * ny and np.all(rest[top, 2] == rest[:, 2].max())
    assert np.isclose(m.extent, (max(nx, ny, nz) - 1) * s, rtol=1e-14)


def _check_coloring(cons, color, order, off):
    """Valid first-fit colouring in index order plus a stable colour-major order."""
    n = len(cons)
    nc = int(color.max()) + 1 if n else 0
    assert len(off) == nc + 1 and off[0] == 0 and off[-1] == n
    for c in range(nc):
        members = order[off[c]:off[c + 1]]
        assert np.all(color[members] == c)
        assert np.all(np.diff(members) > 0)
        verts = cons[members].reshape(-1)
        assert len(np.unique(verts)) == len(verts), "two constraints of one colour share a vertex"
    # first fit: for each constraint and each smaller colour there is an earlier
    # constraint sharing a vertex with that colour
    touching = {}
    for i in range(n):
        seen = set()
        for vtx in cons[i]:
            seen.update(touching.get(int(vtx), ()))
        for c in range(color[i]):
            assert c in seen
        for vtx in cons[i]:
            touching.setdefault(int(vtx), set()).add(int(color[i]))


@pytest.mark.parametrize("shape,ne,nt", [((9, 9, 5), 18, 36), ((17, 17, 9), 18, 37), ((3, 3, 2), None, None)])
def test_coloring_first_fit(shape, ne, nt):
    rest, w, tets = inputs.grid_block(*shape)
    m = oracle.Mesh(rest, w, tets)
    _check_coloring(m.edges, m.ecolor, m.eorder, m.ecol_off)
    _check_coloring(m.tets, m.tcolor, m.torder, m.tcol_off)
    if ne is not None:
        # regression counts of first-fit on these meshes (not paper data)
        assert (m.n_ecol, m.n_tcol) == (ne, nt)


def test_degenerate_and_invalid_meshes_rejected():
    rest, w, tets = inputs.two_tet_mesh()
    bad = tets.copy(); bad[0, 1] = 99
    with pytest.raises(ValueError):
        oracle.Mesh(rest, w, bad)
    dup = tets.copy(); dup[0, 1] = dup[0, 0]
    with pytest.raises(ValueError):
        oracle.Mesh(rest, w, dup)
    flat = rest.copy(); flat[3] = [0.001, 0.001, 0.0]   # tet 0 has zero volume
    with pytest.raises(ValueError):
        oracle.Mesh(flat, w, tets)


# --------------------------------------------------------------------------
# Single projections (Eq. 1, Eqs. 2-3 in XPBD form)
# --------------------------------------------------------------------------

def test_edge_projection_closed_forms():
    d = 0.005
    # equal masses, alpha 0: exact length, midpoint fixed (Eq. 1 with k_s = 1)
    xa, xb = np.array([0.001, 0.002, 0.0]), np.array([0.0071, -0.0013, 0.0009])
    a, b, lam, C = oracle.project_edge(xa, xb, 1000.0, 1000.0, d, 0.0)
    assert np.isclose(np.linalg.norm(a - b), d, rtol=1e-14)
    assert np.allclose((a + b) / 2, (xa + xb) / 2, atol=1e-18)
    assert np.isclose(C, np.linalg.norm(xa - xb) - d, rtol=1e-14)
    # Eq. 1: each vertex moves by w_i/(w_a+w_b) of the violation along x_ab/|x_ab|
    n = (xa - xb) / np.linalg.norm(xa - xb)
    assert np.allclose(a - xa, -0.5 * C * n, atol=1e-18)
    assert np.allclose(b - xb, +0.5 * C * n, atol=1e-18)
    # pinned b
    a, b, lam, C = oracle.project_edge(xa, xb, 1000.0, 0.0, d, 0.0)
    assert np.array_equal(b, xb) and np.isclose(np.linalg.norm(a - b), d, rtol=1e-14)
    # compliance: residual shrinks by alpha~/(w_a+w_b+alpha~), lambda = dlambda
    at = 0.36
    a, b, lam, C = oracle.project_edge(xa, xb, 1000.0, 1000.0, d, at)
    Cn = np.linalg.norm(a - b) - d
    assert np.isclose(Cn, C * at / (2000.0 + at), rtol=1e-9)
    assert np.isclose(lam, -C / (2000.0 + at), rtol=1e-14)
    # lambda carries across iterations: a second pass at the fixed point is a no-op
    a2, b2, lam2, _ = oracle.project_edge(a, b, 1000.0, 1000.0, d, at, lam)
    assert np.allclose(a2, a, atol=1e-18) and np.isclose(lam2, lam, rtol=1e-12)
    # all pinned and no compliance: skipped
    a, b, lam, C = oracle.project_edge(xa, xb, 0.0, 0.0, d, 0.0)
    assert np.array_equal(a, xa) and np.array_equal(b, xb) and lam == 0.0


def _vol(x):
    return np.dot(np.cross(x[1] - x[0], x[2] - x[0]), x[3] - x[0]) / 6.0


def test_tet_projection_restores_volume_with_three_pins():
    s = inputs.CELL
    rest = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], dtype=float)
    V0 = _vol(rest)
    x = 1.1 * rest
    xs, lam, C = oracle.project_tet(x, [0.0, 0.0, 0.0, 1000.0], V0, 0.0)
    assert np.isclose(C, _vol(x) - V0, rtol=1e-14)
    # C is linear in x_d along its gradient, so one projection is exact
    assert abs(_vol(np.array(xs)) - V0) <= 1e-14 * V0
    for i in range(3):
        assert np.array_equal(xs[i], x[i])


def _fd_grad(fun, x, h):
    x = np.array(x, dtype=np.longdouble)
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(3):
            xp = x.copy(); xm = x.copy()
            xp[i, k] += h; xm[i, k] -= h
            g[i, k] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def test_tet_projection_matches_finite_difference_gradient_and_conserves_momenta():
    rng = np.random.default_rng(4)
    s = inputs.CELL
    x = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], dtype=float) + rng.uniform(-1e-3, 1e-3, (4, 3))
    w = np.array([1000.0, 500.0, 2000.0, 1000.0])
    V0 = s**3 / 6
    xs, lam, C = oracle.project_tet(x, w, V0, 0.0)
    dx = np.array(xs) - x

    def vol(xx):
        return np.dot(np.cross(xx[1] - xx[0], xx[2] - xx[0]), xx[3] - xx[0]) / 6

    g = _fd_grad(vol, x, 1e-6).astype(float)
    # XPBD: dx_i = w_i dlambda grad_i C with dlambda = -C / sum w |grad|^2
    dl = -C / np.sum(w * np.sum(g * g, axis=1))
    assert np.allclose(dx, w[:, None] * dl * g, rtol=1e-9, atol=1e-15)
    m = 1.0 / w
    assert np.allclose((m[:, None] * dx).sum(axis=0), 0.0, atol=1e-20)
    assert np.allclose((m[:, None] * np.cross(x, dx)).sum(axis=0), 0.0, atol=1e-22)


# --------------------------------------------------------------------------
# Whole steps (Algorithm 1 with the substep readings)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [1e-2, 1e-4, 1e-6])
def test_static_elongation_equals_m_g_alpha(alpha):
    """A particle hung on one compliant distance constraint settles at the
    elongation m g alpha (the XPBD fixed point with lambda reset per substep)."""
    L = 0.01
    rest = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, -L]])
    w = np.array([0.0, 1.0 / M])
    m = oracle.Mesh(rest, w, np.zeros((0, 4), np.int32), edges=[[0, 1]])
    p = params(alpha_d=alpha, radius=0.0, n_obs=1, action_scale=0.0)
    e = oracle.Env(m, p)
    e.reset(0)
    for _ in range(200):
        e.run(50, actions=np.zeros((50, 3)), want_obs=False)
        x, v, _ = e.state()
        if abs(v[1, 2]) < 1e-14:
            break
    x, v, _ = e.state()
    elong = -x[1, 2] - L
    assert np.isclose(elong, M * G * alpha, rtol=1e-6)
    assert abs(v[1, 2]) < 1e-9


def test_free_fall_matches_symplectic_euler():
    rest = np.array([[0.0, 0.0, 0.0], [0.004, 0.0, 0.0]])
    w = np.array([1.0 / M, 1.0 / M])
    m = oracle.Mesh(rest, w, np.zeros((0, 4), np.int32), edges=[[0, 1]])
    p = params(radius=0.0, n_obs=1, action_scale=0.0)
    e = oracle.Env(m, p)
    e.reset(0)
    n_steps = 7
    e.run(n_steps, actions=np.zeros((n_steps, 3)), want_obs=False)
    x, v, _ = e.state()
    h = p["dt"] / p["substeps"]
    n = n_steps * p["substeps"]
    assert np.allclose(v[:, 2], -G * h * n, rtol=1e-12)
    assert np.allclose(x[:, 2], -G * h * h * n * (n + 1) / 2, rtol=1e-12)
    assert np.allclose(x[:, 0], rest[:, 0], atol=1e-16)


def test_rest_state_is_a_fixed_point_exactly():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), radius=0.0)
    e = oracle.Env(m, p)
    e.reset(1)
    e.run(5, want_obs=False)
    x, v, _ = e.state()
    assert np.array_equal(x, rest) and np.all(v == 0)


def _free_body():
    rest, _, tets = inputs.grid_block(4, 3, 3, pin_bottom=False)
    w = np.full(len(rest), 1.0 / M)
    return rest, w, tets


def test_free_body_conserves_linear_momentum():
    rest, w, tets = _free_body()
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), radius=0.0, n_obs=4, iterations=2)
    e = oracle.Env(m, p)
    e.reset(2)
    rng = np.random.default_rng(9)
    x0 = inputs.perturbed_positions(rest, 1e-3, 5)
    v0 = rng.normal(0, 0.05, rest.shape)
    e.set_state(x=x0, v=v0)
    P0 = (v0 / w[:, None]).sum(axis=0)
    com0 = (x0 / w[:, None]).sum(axis=0) / (1 / w).sum()
    n_steps = 20
    e.run(n_steps, want_obs=False)
    x, v, _ = e.state()
    P = (v / w[:, None]).sum(axis=0)
    assert np.allclose(P, P0, atol=1e-14)
    com = (x / w[:, None]).sum(axis=0) / (1 / w).sum()
    vcom = P0 / (1 / w).sum()
    assert np.allclose(com, com0 + n_steps * p["dt"] * vcom, atol=1e-13)
    assert not np.allclose(x, x0 + n_steps * p["dt"] * v0, atol=1e-6)  # constraints did act


def test_free_body_is_rotation_equivariant():
    rest, w, tets = _free_body()
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), radius=0.0, n_obs=4)
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    x0 = inputs.perturbed_positions(rest, 1e-3, 8)
    v0 = rng.normal(0, 0.05, rest.shape)
    outs = []
    for R in (np.eye(3), q):
        e = oracle.Env(m, p)
        e.reset(0)
        e.set_state(x=x0 @ R.T, v=v0 @ R.T)
        e.run(5, want_obs=False)
        outs.append(e.state()[0])
    assert np.allclose(outs[0] @ q.T, outs[1], atol=1e-12)


def _brute_force_step(rest, w, tets, x, v, c, p, action, n_obs_ok=True):
    """Independent loop-per-constraint re-implementation of one step: edges and
    colours recomputed here, every gradient by central finite differences of C
    in long double, then the XPBD update, sphere push-out and velocity update."""
    L = np.longdouble
    rest = rest.astype(L); x = x.astype(L); v = v.astype(L); c = c.astype(L)
    tets = [list(t) for t in tets]
    for t in tets:  # orient (vertices 2, 3 swapped if the rest volume is negative)
        if _vol(rest[t]) < 0:
            t[2], t[3] = t[3], t[2]
    edges = sorted({tuple(sorted((t[a], t[b]))) for t in tets for a, b in itertools.combinations(range(4), 2)})

    def first_fit(cons):
        col, used = [], {}
        for cc in cons:
            k = 0
            while any(k in used.get(vv, ()) for vv in cc):
                k += 1
            col.append(k)
            for vv in cc:
                used.setdefault(vv, set()).add(k)
        return col

    ecol, tcol = first_fit(edges), first_fit(tets)
    order = [("e", i) for c_ in range(max(ecol) + 1) for i in range(len(edges)) if ecol[i] == c_]
    order += [("t", i) for c_ in range(max(tcol) + 1) for i in range(len(tets)) if tcol[i] == c_]
    d = [np.sqrt(np.sum((rest[a] - rest[b]) ** 2)) for a, b in edges]
    V0 = [_vol(rest[t]) for t in tets]
    lo = np.array([rest[:, 0].min() - L(p["margin_xy"]), rest[:, 1].min() - L(p["margin_xy"]),
                   rest[:, 2].max() - L(p["margin_below"])])
    hi = np.array([rest[:, 0].max() + L(p["margin_xy"]), rest[:, 1].max() + L(p["margin_xy"]),
                   rest[:, 2].max() + L(p["margin_above"])])
    c = np.minimum(np.maximum(c + L(p["action_scale"]) * np.asarray(action, dtype=L), lo), hi)
    h = L(p["dt"]) / p["substeps"]
    g = np.asarray(p["gravity"], dtype=L)
    w = w.astype(L)
    pushes = 0
    for _ in range(p["substeps"]):
        xprev = x.copy()
        free = w > 0
        v[free] += h * g
        x[free] += h * v[free]
        lam = {}
        for _it in range(p["iterations"]):
            for kind, i in order:
                if kind == "e":
                    idx = list(edges[i]); at = L(p["alpha_d"]) / (h * h)
                    fun = lambda xx, i=i: np.sqrt(np.sum((xx[0] - xx[1]) ** 2)) - d[i]  # noqa: E731
                else:
                    idx = tets[i]; at = L(p["alpha_v"]) / (h * h)
                    fun = lambda xx, i=i: _vol(xx) - V0[i]  # noqa: E731
                xl = x[idx]
                C = fun(xl)
                gr = _fd_grad(fun, xl, L(1e-9))
                wl = w[idx]
                lm = lam.get((kind, i), L(0))
                dl = (-C - at * lm) / (np.sum(wl * np.sum(gr * gr, axis=1)) + at)
                x[idx] = xl + wl[:, None] * dl * gr
                lam[(kind, i)] = lm + dl
        r = L(p["radius"])
        for i in range(len(x)):
            if w[i] == 0:
                continue
            dv = x[i] - c
            n = np.sqrt(np.sum(dv * dv))
            if n < r:
                x[i] = c + r * dv / n
                pushes += 1
        v = (x - xprev) / h
    return x.astype(float), v.astype(float), c.astype(float), pushes


@pytest.mark.parametrize("iterations", [1, 2])
def test_two_tet_mesh_matches_brute_force(iterations):
    rest, w, tets = inputs.two_tet_mesh()
    w = w.copy(); w[0] = 0.0; w[2] = 250.0    # one pinned vertex, one heavy one
    p = params(n_obs=2, iterations=iterations, alpha_d=1e-4, alpha_v=1e-9)
    m = oracle.Mesh(rest, w, tets)
    e = oracle.Env(m, p)
    e.reset(0)
    x0 = inputs.perturbed_positions(rest, 4e-4, 1, inv_mass=w)
    v0 = np.random.default_rng(2).normal(0, 0.02, rest.shape); v0[w == 0] = 0
    e.set_state(x=x0, v=v0)
    _, _, c0 = e.state()
    action = np.array([1.0, 1.0, -1.0])   # drives the sphere into vertex 4
    e.step(action)
    x, v, c = e.state()
    xb, vb, cb, pushes = _brute_force_step(rest, w, tets, x0, v0, c0, p, action)
    assert np.allclose(c, cb, atol=1e-15)
    assert pushes >= 1
    assert np.max(np.abs(x - xb)) <= 1e-9 * m.extent
    assert np.max(np.abs(v - vb)) <= 1e-9 * m.extent / (p["dt"] / p["substeps"])


def test_sphere_collision_projects_inside_vertices_only():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), iterations=0, substeps=1, radius=7e-3)
    e = oracle.Env(m, p)
    e.reset(0)
    x0 = inputs.perturbed_positions(rest, 1e-3, 4, inv_mass=w)
    c = np.array([0.0012, -0.0031, 0.0175])
    e.set_state(x=x0, v=np.zeros_like(x0), c=c)
    e.step(np.zeros(3))
    x, _, c1 = e.state()
    assert np.array_equal(c1, c)
    dist0 = np.linalg.norm(x0 - c, axis=1)
    inside = (dist0 < p["radius"]) & (w > 0)
    assert inside.sum() >= 3
    assert np.array_equal(x[~inside], x0[~inside])
    assert np.allclose(np.linalg.norm(x[inside] - c, axis=1), p["radius"], rtol=1e-15)
    # pushed along the centre-to-vertex direction
    dirs0 = (x0[inside] - c) / dist0[inside, None]
    dirs1 = (x[inside] - c) / p["radius"]
    assert np.allclose(dirs0, dirs1, atol=1e-13)
    assert e.ints()["contacts"].tolist() == np.nonzero(inside)[0].tolist()


def test_reset_obs_reward_and_termination():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), radius=0.0, w_l=-1.0, w_d=-10.0, w_s=100.0, max_steps=3)
    e = oracle.Env(m, p)
    seed, env = 21, 6
    e.reset(seed, env)
    info = e.ints()
    top = m.top
    assert info["obs_ids"].tolist() == top[oracle.sample_indices(seed, env, len(top), 64)].tolist()
    assert info["target"] == top[oracle.target_index(seed, env, len(top))]
    _, _, c = e.state()
    s = inputs.CELL
    assert np.allclose(c, [0.0, 0.0, rest[:, 2].max() + p["radius"]], atol=1e-18)
    lo, hi = e.tool_box()
    assert np.allclose(lo, [rest[:, 0].min() - 2 * s, rest[:, 1].min() - 2 * s, rest[:, 2].max() - s])
    assert np.allclose(hi, [rest[:, 0].max() + 2 * s, rest[:, 1].max() + 2 * s, rest[:, 2].max() + 6 * s])
    obs, R, done = e.step(np.zeros(3))
    assert np.array_equal(obs[:3], c)
    assert np.array_equal(obs[3:].reshape(-1, 3), rest[info["obs_ids"]])
    l0 = np.linalg.norm(c - rest[info["target"]])
    assert np.isclose(R, -l0, rtol=1e-14) and done == 0      # d = 0, s = 0
    # move the tool within 3 mm of the target: success flag, reward and done
    tgt = rest[info["target"]]
    e.set_state(c=tgt + np.array([0.0, 0.0, 0.002]))
    obs, R, done = e.step(np.zeros(3))
    assert done == 1
    assert np.isclose(R, -0.002 + (-10.0) * (0.002 - l0) + 100.0, rtol=1e-12)
    e.set_state(c=c)
    _, _, done = e.step(np.zeros(3))
    assert done == 1                                             # step limit reached


def test_tool_is_clamped_to_its_box():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(gravity=(0.0, 0.0, 0.0), radius=0.0)
    e = oracle.Env(m, p)
    e.reset(0)
    lo, hi = e.tool_box()
    e.run(60, actions=np.tile([1.0, -1.0, 1.0], (60, 1)), want_obs=False)
    _, _, c = e.state()
    assert np.array_equal(c, [hi[0], lo[1], hi[2]])
