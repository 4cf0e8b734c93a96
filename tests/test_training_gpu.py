"""Training of the warm-start network on the tensor cores.

The gradient of the weighted mean squared error computed by the fused
tcgen05 training kernel (BF16 operands, FP32 accumulation) is compared with
the FP64 oracle's backward pass (oracle/mlp.py, pinned by finite differences)
evaluated with BF16 rounding at the kernel's rounding points, element by
element: |g_gpu - g_ref| <= 1e-2 x the largest |g_ref| of the parameter block
(FP32 accumulation order, and the occasional bfloat16 rounding flip of one
dY / dZ entry that it causes, 2^-8 of one term). Against the unrounded FP64
gradient the per-block relative Frobenius error must stay below 6e-2 with a
cosine above 0.998. The Adam kernel and the BF16 repacking are compared with
the oracle's Adam (Kingma & Ba 2015) over five steps of seeded gradients, the
device normalisation with the oracle's, and training must reduce the loss of
a regression onto a fixed teacher network.
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs
from sim_helpers import grid, make_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def _setup(rows, seed, zero_frac=0.1):
    rng = np.random.default_rng(seed)
    p = oracle.mlp_init(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.05, p[k].shape)
    in_mean, in_std = rng.normal(0, 1e-3, 15), rng.uniform(1e-3, 3e-3, 15)
    out_mean, out_std = rng.normal(0, 1e-6, 3), rng.uniform(1e-6, 3e-6, 3)
    F = np.zeros((rows, 16), np.float32)
    F[:, :15] = rng.normal(size=(rows, 15)) * in_std + in_mean
    T = np.zeros((rows, 4), np.float32)
    T[:, :3] = rng.normal(size=(rows, 3)) * out_std + out_mean
    w = (rng.uniform(size=rows) > zero_frac).astype(np.float32)
    return p, (in_mean, in_std, out_mean, out_std), F, T, w


def _bf16_reference_gradient(p, Xn, Tn):
    """The oracle's backward pass with BF16 rounding applied where the kernel
    rounds: inputs, weights, hidden activations, dY, dZ2, dZ1 (bias gradients
    and the loss use the unrounded values)."""
    bf = oracle.bf16_round
    W1, W2, W3 = bf(p["W1"]), bf(p["W2"]), bf(p["W3"])
    Xb = bf(Xn)
    h1 = np.maximum(Xb @ W1.T + p["b1"], 0)
    H1 = bf(h1)
    h2 = np.maximum(H1 @ W2.T + p["b2"], 0)
    H2 = bf(h2)
    y = H2 @ W3.T + p["b3"]
    g = 2.0 * (y - Tn) / (3 * len(Xn))
    gb = bf(g)
    dz2 = (gb @ W3) * (h2 > 0)
    dz2b = bf(dz2)
    dz1 = (dz2b @ W2) * (h1 > 0)
    dz1b = bf(dz1)
    return {"W3": gb.T @ H2, "b3": g.sum(0), "W2": dz2b.T @ H1, "b2": dz2.sum(0),
            "W1": dz1b.T @ Xb, "b1": dz1.sum(0)}


@pytest.mark.parametrize("rows", [300, 5000])
def test_tensor_core_gradient_matches_fp64_oracle(rows):
    p, norm, F, T, w = _setup(rows, 4)
    sim = make_sim([grid((3, 3, 2))], inputs.default_params(n_obs=4), 1)
    sim.set_network(p, *norm)
    g, loss = sim.network_gradient(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(),
                                   torch.from_numpy(w).cuda(), float(w.sum()))
    sel = w > 0
    Xn = (F[sel, :15].astype(np.float64) - norm[0]) / norm[1]
    Tn = (T[sel, :3].astype(np.float64) - norm[2]) / norm[3]
    y, cache = oracle.mlp_forward(p, Xn)
    ref = oracle.mlp_backward(p, cache, y, Tn)
    ref_loss = np.sum((y - Tn) ** 2)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    refb = _bf16_reference_gradient(p, Xn, Tn)
    for k in KEYS:
        a, b, c = g[k].reshape(-1), ref[k].reshape(-1), refb[k].reshape(-1)
        # tight, element by element: same rounding points, FP32 versus FP64
        # accumulation (a wrong column or row of a weight block fails here)
        err = np.abs(a - c).max() / np.abs(c).max()
        assert err <= 1e-2, (k, err)
        # loose: against the unrounded FP64 gradient (BF16 rounding compounds
        # through dY, dZ2 and dZ1 before reaching the first layer)
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert rel <= 6e-2 and cos > 0.998, (k, rel, cos)


def test_adam_steps_fit_a_teacher_network():
    rows = 20000
    p, norm, F, _, w = _setup(rows, 6, zero_frac=0.0)
    teacher = oracle.mlp_init(99)
    Xn = (F[:, :15].astype(np.float64) - norm[0]) / norm[1]
    yt, _ = oracle.mlp_forward(teacher, Xn)
    T = np.zeros((rows, 4), np.float32)
    T[:, :3] = yt * norm[3] + norm[2]
    sim = make_sim([grid((3, 3, 2))], inputs.default_params(n_obs=4), 1)
    sim.set_network(p, *norm)
    Fd, Td, wd = torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(w).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for it in range(300):
        sim.train_network(Fd, Td, wd, float(w.sum()), 2e-3, loss)
        if it % 50 == 0 or it == 299:
            losses.append(float(loss.item()) / (3 * w.sum()))
    sim.sync()
    assert losses[-1] < 0.2 * losses[0], losses
    q = sim.get_network()
    assert not np.allclose(q["W2"], p["W2"])
    # the trained master weights reproduce the loss the kernel reported
    y, _ = oracle.mlp_forward(q, Xn)
    mse = np.mean((y - yt) ** 2)
    assert mse < 0.3 * losses[0]


def test_adam_steps_and_bf16_repack_match_the_oracle():
    """Five Adam steps (lr 1e-3) of the float32 masters on seeded gradients
    through ffsrl_network_adam_step, the kernel that ffsrl_train_network runs
    after its gradient, against oracle.adam_step in FP64 from the same start:
    masters within 2e-6 (float32 rounding of five updates of size <= lr), and
    the network the repacked BF16 tiles compute equal to the oracle's BF16
    network of the oracle's masters (the forward bar of the network test)."""
    rows = 700
    p, norm, F, _, _ = _setup(rows, 8)
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    sim = make_sim([grid((3, 3, 2))], inputs.default_params(n_obs=4), 1)
    sim.set_network(p, *norm)
    rng = np.random.default_rng(21)
    q = {k: v.copy() for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(val) for k, val in p.items()}
    lr = 1e-3
    for t in range(1, 6):
        gk = {k: rng.normal(0, 1e-2, p[k].shape).astype(np.float32).astype(np.float64) for k in KEYS}
        gk["W2"][3, :] = 0.0     # exact zeros: no update
        flat = np.concatenate([gk[k].reshape(-1) for k in KEYS]).astype(np.float32)
        sim.network_adam_step(torch.from_numpy(flat).cuda(), lr)
        oracle.adam_step(q, gk, m, v, t, lr=lr)
    got = sim.get_network()
    for k in KEYS:
        err = np.abs(got[k] - q[k]).max()
        assert err <= 2e-6, (k, err)
        moved = np.abs(got[k] - p[k]).max()
        assert moved > 1e-3, k   # five steps of about lr each
    assert np.array_equal(got["W2"][3, :], p["W2"][3, :].astype(np.float32))
    out = sim.network_forward(torch.from_numpy(F).cuda())
    sim.sync()
    net = oracle.Net.from_params(q, *norm, bf16=True)
    ref = oracle.net_forward(net, F[:, :15].astype(np.float64))
    e = np.abs(out.cpu().numpy()[:, :3] - ref) / norm[3]
    assert e.max() <= 3e-2 and e.mean() <= 2e-3, (e.max(), e.mean())


@pytest.mark.parametrize("rows", [1, 1000, 300_000])
def test_device_normalisation_matches_the_oracle(rows):
    """ffsrl_network_normalisation (two passes in double on the device)
    against oracle.normalisation on the same float32 rows: the float32 results
    within 1e-6 relative (of the std for the means) plus their own float32
    rounding; rows of zero weight carry huge values that must not count."""
    rng = np.random.default_rng(rows)
    F = np.zeros((rows, 16), np.float32)
    F[:, :15] = rng.normal(size=(rows, 15)) * rng.uniform(1e-4, 1e-2, 15) + rng.normal(0, 1e-3, 15)
    F[:, 5] = 0.25                       # a column without spread
    T = np.zeros((rows, 4), np.float32)
    T[:, :3] = rng.normal(size=(rows, 3)) * 1e-5 + 1e-6
    w = (rng.uniform(size=rows) > 0.2).astype(np.float32)
    w[0] = 1.0
    F[w == 0, :15] = 1e6
    sim = make_sim([grid((3, 3, 2))], inputs.default_params(n_obs=4), 1)
    got = sim.network_normalisation(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(),
                                    torch.from_numpy(w).cuda())
    want = oracle.normalisation(F.astype(np.float64), T.astype(np.float64), w)
    for name, g, r in zip(("in_mean", "in_std", "out_mean", "out_std"), got, want):
        scale = want[1] if name == "in_mean" else want[3] if name == "out_mean" else r
        # double sums, one float32 rounding of the result
        assert np.all(np.abs(g - r) <= 1e-6 * np.abs(scale) + 2.0 ** -23 * np.abs(r)), name
    assert got[1][5] == 1.0 and got[0][5] == 0.25
    from paper_2503_18616_gb300 import ffsrl
    with pytest.raises(ffsrl.FfsrlError):
        sim.network_normalisation(torch.from_numpy(F).cuda(), torch.from_numpy(T).cuda(),
                                  torch.zeros(rows, dtype=torch.float32, device="cuda"))
