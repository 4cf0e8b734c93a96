"""Pins of the FP64 warm-start network oracle (oracle/mlp.py).

The network is not in the FF-SRL paper; it is the per-vertex 15-64-64-3 ReLU
perceptron of the learned warm-start. Its oracle is pinned by central
finite differences of the loss, by closed forms of degenerate networks, by
Adam's first-step closed form (Kingma & Ba, ICLR 2015, Algorithm 1), and by
exact bfloat16 rounding cases.
"""
import numpy as np

import oracle


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, oracle.N_IN)), rng.normal(size=(n, oracle.N_OUT))


def test_backward_matches_central_differences():
    p = oracle.mlp_init(3)
    for k in p:
        if k.startswith("b"):
            p[k] = np.random.default_rng(len(k)).normal(0, 0.1, p[k].shape)
    F, T = _batch(17, 1)
    y, cache = oracle.mlp_forward(p, F)
    g = oracle.mlp_backward(p, cache, y, T)
    rng = np.random.default_rng(5)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = oracle.mlp_loss(oracle.mlp_forward(p, F)[0], T)
            flat[idx] = old - h
            lm = oracle.mlp_loss(oracle.mlp_forward(p, F)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert np.isclose(g[name].reshape(-1)[idx], fd, rtol=1e-5, atol=1e-9), name


def test_bias_only_network_closed_form():
    p = {k: np.zeros_like(v) for k, v in oracle.mlp_init(0).items()}
    p["b3"] = np.array([0.5, -1.0, 2.0])
    F, T = _batch(8, 2)
    y, cache = oracle.mlp_forward(p, F)
    assert np.array_equal(y, np.tile(p["b3"], (8, 1)))
    g = oracle.mlp_backward(p, cache, y, T)
    assert np.allclose(g["b3"], 2.0 * (p["b3"] - T).mean(axis=0) / 3.0)
    for k in ("W1", "W2", "W3", "b1", "b2"):
        assert np.all(g[k] == 0)   # every ReLU is closed at zero input


def test_linear_regime_equals_matrix_product():
    # with every pre-activation positive the network is the product of the layers
    p = oracle.mlp_init(1)
    p["b1"] = np.full(64, 100.0)
    p["b2"] = np.full(64, 1000.0)
    p["W2"] = np.abs(p["W2"])
    F, _ = _batch(5, 3)
    y, _ = oracle.mlp_forward(p, F)
    ref = ((F @ p["W1"].T + p["b1"]) @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"]
    assert np.allclose(y, ref, rtol=1e-12)


def test_adam_first_step_is_signed_learning_rate():
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.3, -4.0, 1e-3])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    oracle.adam_step(p, g, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(p["a"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=1e-14)


def test_bf16_rounding_cases():
    cases = {
        1.0: 1.0,
        1.0 + 2.0**-8: 1.0,                    # tie, rounds to even
        1.0 + 3 * 2.0**-8: 1.0 + 2.0**-6,      # tie, rounds up to even
        1.0 + 2.0**-7: 1.0 + 2.0**-7,          # exactly representable
        -3.0 - 2.0**-9: -3.0,
        65280.0: 65280.0,
    }
    for x, want in cases.items():
        assert oracle.bf16_round(np.array([x]))[0] == want, x
