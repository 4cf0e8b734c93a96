"""Pins of the oracle's surrogate-assisted substep (learned warm-start).

The warm-start is not in the FF-SRL paper; its oracle is pinned by limiting
cases that reduce it to the plain XPBD step, by invariants of its features,
by a closed form of the residual, and by agreement of the C network with the
separately pinned numpy network (oracle/mlp.py).
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs


def _env(shape=(5, 4, 3), **over):
    m = oracle.Mesh(*inputs.grid_block(*shape))
    p = inputs.default_params(n_obs=4, **over)
    e = oracle.Env(m, p)
    e.reset(3)
    return m, p, e


def _zero_net():
    return oracle.Net.from_params({k: np.zeros_like(v) for k, v in oracle.mlp_init(0).items()})


def test_c_network_equals_numpy_network():
    p = oracle.mlp_init(5)
    rng = np.random.default_rng(1)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    mean, std = rng.normal(size=15), rng.uniform(0.5, 2.0, 15)
    omean, ostd = rng.normal(size=3), rng.uniform(0.5, 2.0, 3)
    net = oracle.Net.from_params(p, mean, std, omean, ostd)
    F = rng.normal(size=(40, 15))
    got = oracle.net_forward(net, F)
    y, _ = oracle.mlp_forward(p, (F - mean) / std)
    assert np.allclose(got, y * ostd + omean, rtol=1e-12, atol=1e-12)
    # with bfloat16 rounding of inputs, weights and hidden activations
    netb = oracle.Net.from_params(p, mean, std, omean, ostd, bf16=True)
    pb = {k: (oracle.bf16_round(v) if k.startswith("W") else v) for k, v in p.items()}
    Fb = oracle.bf16_round((F - mean) / std)
    h1 = oracle.bf16_round(np.maximum(Fb @ pb["W1"].T + pb["b1"], 0))
    h2 = oracle.bf16_round(np.maximum(h1 @ pb["W2"].T + pb["b2"], 0))
    yb = h2 @ pb["W3"].T + pb["b3"]
    assert np.allclose(oracle.net_forward(netb, F), yb * ostd + omean, rtol=1e-12, atol=1e-12)


def test_features_at_rest_and_under_rigid_motion():
    m, p, e = _env(gravity=(0.0, 0.0, 0.0))
    F = e.features()
    x, v, c = e.state()
    assert np.all(F[:, 0:6] == 0) and np.all(F[:, 9:12] == 0)
    assert np.allclose(F[:, 12:15], x - c, atol=1e-18)
    # a rigid translation with velocity u: displacement shifts, velocity
    # features are u and the 1-ring velocity offsets vanish; 1-ring position
    # offsets do not change
    u = np.array([0.03, -0.01, 0.02])
    shift = np.array([1e-3, 2e-3, -5e-4])
    e.set_state(x=x + shift, v=np.tile(u, (m.V, 1)) * (m.inv_mass > 0)[:, None])
    G = e.features()
    h = p["dt"] / p["substeps"]
    free = m.inv_mass > 0
    assert np.allclose(G[free, 3:6], u, atol=1e-15)
    assert np.allclose(G[free, 0:3], shift + h * u, atol=1e-15)
    # every 1-ring position offset is the rest one plus the mean relative motion
    edges = m.edges
    nb = [[] for _ in range(m.V)]
    for a, b in edges:
        nb[a].append(b)
        nb[b].append(a)
    for i in range(m.V):
        if free[i] and all(free[j] for j in nb[i]):
            assert np.allclose(G[i, 6:9], F[i, 6:9], atol=1e-15)
            assert np.allclose(G[i, 9:12], 0, atol=1e-15)


def test_residual_closed_forms():
    m, p, e = _env()
    assert e.residual() == 0.0
    x, _, _ = e.state()
    eps = 1e-3
    e.set_state(x=x * (1 + eps))   # uniform scaling about the origin
    assert np.isclose(e.residual(), (1 + eps) ** 3 - 1, rtol=1e-9)


def test_zero_network_without_fallback_is_the_one_iteration_step():
    for seed in (0, 1):
        m, p, e1 = _env(iterations=1)
        _, _, e2 = _env(iterations=1)
        e1.reset(seed)
        e2.reset(seed)
        for _ in range(6):
            o1, r1, d1 = e1.step()
            o2, r2, d2, fb = e2.step_surrogate(_zero_net(), threshold=np.inf, n_full=10)
            assert fb == 0
            assert np.array_equal(o1, o2) and r1 == r2
        assert np.array_equal(e1.state()[0], e2.state()[0])


@pytest.mark.parametrize("n_full", [3, 10])
def test_always_falling_back_is_the_full_solve(n_full):
    m, p, e1 = _env(iterations=n_full)
    _, _, e2 = _env(iterations=1)
    net = oracle.Net.from_params(oracle.mlp_init(2), out_std=np.full(3, 1e-4))   # a poor network
    for _ in range(5):
        o1, _, _ = e1.step()
        o2, _, _, fb = e2.step_surrogate(net, threshold=-1.0, n_full=n_full)
        assert fb == p["substeps"]
        assert np.array_equal(o1, o2)
    assert np.array_equal(e1.state()[0], e2.state()[0])
    assert np.array_equal(e1.state()[1], e2.state()[1])


def test_recorded_targets_reproduce_the_full_solve():
    m, p, e1 = _env(iterations=10)
    _, _, e2 = _env(iterations=1)
    for _ in range(3):
        x0, v0, _ = e2.state()
        F, T = e2.step_record(n_full=10)
        e1.step()
        assert F.shape == (p["substeps"], m.V, 15) and T.shape == (p["substeps"], m.V, 3)
    assert np.array_equal(e1.state()[0], e2.state()[0])
    # pinned vertices never move, so their targets are zero
    assert np.all(T[:, m.inv_mass == 0] == 0)
    assert np.abs(T).max() > 0


def test_more_iterations_leave_a_smaller_residual():
    """The premise of the warm-start: the full solve ends closer to the
    constraint manifold than one iteration from the bare prediction."""
    _, _, e_one = _env(iterations=1)
    e_one.step()
    _, _, e_ref = _env(iterations=10)
    e_ref.step()
    assert e_ref.residual() < e_one.residual()


def test_one_ring_features_closed_form_on_the_top_face():
    """F[:, 6:9] (and 9:12) against the grid geometry. The five-tet split puts
    an edge on every axis-aligned grid segment and on the one face diagonal of
    each cell face that joins its two corners with an odd coordinate sum. On
    the top face of a 5x5x3 block (spacing D, gravity off) that gives:
      - vertex (2,2,2), even: neighbours +-x, +-y and -z: offset (0, 0, -D/5);
      - vertex (1,2,2), odd: five axis neighbours, four diagonals in the top
        face and four going down: offset (0, 0, -5D/13);
      - corner (0,0,2), even: +x, +y, -z: offset (D, D, -D)/3.
    A 1-ring mean that counted the vertex itself would give -D/6, -5D/14 and
    D/4. With velocities v_z = k z (k a constant) the velocity offsets are k
    times the z position offsets, and the predicted positions move by h v."""
    D = inputs.CELL
    m = oracle.Mesh(*inputs.grid_block(5, 5, 3))
    p = inputs.default_params(n_obs=4, gravity=(0.0, 0.0, 0.0))
    e = oracle.Env(m, p)
    e.reset(1)
    F = e.features()
    vid = lambda i, j, k: (k * 5 + j) * 5 + i  # noqa: E731
    cases = {vid(2, 2, 2): (0.0, 0.0, -D / 5), vid(1, 2, 2): (0.0, 0.0, -5 * D / 13),
             vid(0, 0, 2): (D / 3, D / 3, -D / 3)}
    for i, want in cases.items():
        assert np.allclose(F[i, 6:9], want, rtol=1e-12, atol=1e-18), i
    # velocity field v = (0, 0, k z) on the free vertices
    kz = 2.0
    x, _, _ = e.state()
    v = np.zeros_like(x)
    v[:, 2] = kz * x[:, 2] * (m.inv_mass > 0)
    e.set_state(v=v)
    G = e.features()
    h = p["dt"] / p["substeps"]
    for i, want in cases.items():
        # z offsets scale by (1 + h k) for positions and by k for velocities
        # (every neighbour here is free: the bottom layer is two cells below)
        assert np.allclose(G[i, 6:9], np.array(want) * [1, 1, 1 + h * kz], rtol=1e-12, atol=1e-18), i
        assert np.allclose(G[i, 9:12], [0.0, 0.0, kz * want[2]], rtol=1e-12, atol=1e-18), i


def test_surrogate_step_refuses_the_grasper():
    """The warm-start is defined with the sphere tool (the network's features
    have no grasp or face terms), as on the GPU, which refuses it too."""
    m = oracle.Mesh(*inputs.grid_block(5, 4, 3))
    p = inputs.default_params(n_obs=4, tool_model=1)
    e = oracle.Env(m, p)
    e.reset(0)
    with pytest.raises(ValueError):
        e.step_surrogate(_zero_net(), threshold=np.inf, n_full=10)
    with pytest.raises(ValueError):
        e.step_record(n_full=10)


def test_recorded_residuals_are_the_checked_ones():
    """The per-substep residuals the surrogate step reports are those the
    threshold decision saw: with the threshold between two of them, exactly
    the substeps above it fall back."""
    m, p, e1 = _env(iterations=1)
    net = oracle.Net.from_params(oracle.mlp_init(2), out_std=np.full(3, 1e-6))
    r = np.zeros(p["substeps"])
    e1.step_surrogate(net, threshold=np.inf, n_full=5, residuals=r)
    assert np.all(r > 0)
    thr = float(np.median(r))
    _, _, e2 = _env(iterations=1)
    r2 = np.zeros(p["substeps"])
    _, _, _, fb = e2.step_surrogate(net, threshold=thr, n_full=5, residuals=r2)
    assert r2[0] == r[0]                        # the same first substep
    assert fb == int(np.sum(r2 > thr)) and 0 < fb < p["substeps"]


def test_threshold_reading_for_nan_and_infinity():
    """A threshold of +inf never falls back; a finite one falls back unless the
    residual is at most it, so a network that returns NaN makes every substep
    fall back to the full solve (which is then the plain full-solve step)."""
    p = oracle.mlp_init(0)
    p["b3"] = np.array([np.nan, 0.0, 0.0])
    net = oracle.Net.from_params(p)
    m, prm, e1 = _env(iterations=10)
    _, _, e2 = _env(iterations=1)
    for _ in range(2):
        e1.step()
        _, _, _, fb = e2.step_surrogate(net, threshold=1e9, n_full=10)
        assert fb == prm["substeps"]
    assert np.array_equal(e1.state()[0], e2.state()[0])
    _, _, e3 = _env(iterations=1)
    _, _, _, fb = e3.step_surrogate(net, threshold=np.inf, n_full=10)
    assert fb == 0 and np.isnan(e3.state()[0]).any()
