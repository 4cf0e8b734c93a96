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


def test_adam_constant_gradient_closed_form():
    """For a constant gradient g the moments are m_t = g (1 - b1^t) and
    v_t = g^2 (1 - b2^t), so the bias-corrected step is lr g / (|g| + eps) at
    every t; a swapped b1/b2 or a wrong bias-correction power fails at t = 2, 3."""
    g0 = np.array([0.3, -4.0, 1e-3, 2.5e-6])
    p0 = np.array([1.0, -2.0, 3.0, 0.5])
    lr, eps = 0.01, 1e-8
    p = {"a": p0.copy()}
    m = {"a": np.zeros(4)}
    v = {"a": np.zeros(4)}
    for t in (1, 2, 3):
        oracle.adam_step(p, {"a": g0.copy()}, m, v, t, lr=lr, eps=eps)
        want = p0 - t * lr * g0 / (np.abs(g0) + eps)
        assert np.allclose(p["a"], want, rtol=1e-13, atol=1e-15), t
        assert np.allclose(m["a"], g0 * (1 - 0.9 ** t), rtol=1e-13)
        assert np.allclose(v["a"], g0 ** 2 * (1 - 0.999 ** t), rtol=1e-13)


def test_adam_two_steps_by_hand():
    """Gradients g1 = 1 then g2 = -1 (b1 0.9, b2 0.999): m1 = 0.1, v1 = 0.001,
    so the first step is lr; m2 = 0.09 - 0.1 = -0.01 and v2 = 0.000999 + 0.001
    = 0.001999 = 1 - 0.999^2, so m2_hat = -0.01 / 0.19 = -1/19 and v2_hat = 1:
    the second step is -lr/19. With g2 = 3 instead: m2 = 0.39, m2_hat = 39/19,
    v2 = 0.009999, v2_hat = 9999/1999."""
    lr = 0.01
    for g2, step2 in ((-1.0, -lr / 19.0), (3.0, lr * (39.0 / 19.0) / np.sqrt(9999.0 / 1999.0))):
        p = {"a": np.array([0.25])}
        m = {"a": np.zeros(1)}
        v = {"a": np.zeros(1)}
        oracle.adam_step(p, {"a": np.array([1.0])}, m, v, 1, lr=lr, eps=0.0)
        assert np.isclose(p["a"][0], 0.25 - lr, rtol=1e-14)
        oracle.adam_step(p, {"a": np.array([g2])}, m, v, 2, lr=lr, eps=0.0)
        assert np.isclose(p["a"][0], 0.25 - lr - step2, rtol=1e-13), g2


def test_normalisation_closed_forms():
    """Columns taking two values a and b equally often have mean (a + b)/2
    and standard deviation |a - b|/2; a constant column gets std 1; rows of
    zero weight do not count; scaling a column by s scales its mean by s and
    its std by |s|."""
    n = 64
    a = np.linspace(-1, 2, 15)
    b = a + np.arange(1, 16)
    F = np.zeros((2 * n + 3, 16))
    F[:n, :15] = a
    F[n:2 * n, :15] = b
    F[2 * n:, :15] = 1e6            # zero-weight rows
    F[:, 7] = 3.0                   # constant column
    T = np.zeros((2 * n + 3, 4))
    T[:n, :3] = [1.0, -2.0, 5.0]
    T[n:2 * n, :3] = [3.0, -2.0, -5.0]
    w = np.ones(2 * n + 3)
    w[2 * n:] = 0.0
    im, isd, om, osd = oracle.normalisation(F, T, w)
    want_m = (a + b) / 2
    want_s = np.abs(b - a) / 2
    want_m[7], want_s[7] = 3.0, 1.0
    assert np.allclose(im, want_m, rtol=1e-14) and np.allclose(isd, want_s, rtol=1e-14)
    assert np.allclose(om, [2.0, -2.0, 0.0]) and np.allclose(osd, [1.0, 1.0, 5.0])
    s = -2.5
    F2 = F.copy()
    F2[:, 3] *= s
    im2, isd2, _, _ = oracle.normalisation(F2, T, w)
    assert np.isclose(im2[3], s * im[3]) and np.isclose(isd2[3], abs(s) * isd[3])
