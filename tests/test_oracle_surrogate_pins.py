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
