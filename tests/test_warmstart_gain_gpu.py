"""What the trained warm-start network gains over the method without it.

The network is trained on the device by the library's own kernels
(surrogate.train: recording on the full 10-iteration solve, device
normalisation, tensor-core forward and backward, Adam), on a batch of the
9x9x5 block. Then, from the same reset, the warm-start step (network + one
iteration per substep, no fallback) and the plain step with the same single
iteration advance the same envs, and both are compared with the FP64 oracle
running the full solve, the accuracy the network was trained to reach:

  * the warm-start's largest vertex error must be at most half the plain
    step's (the measured ratio is printed);
  * the warm-start step with the trained weights must match the oracle's
    surrogate step with the same weights and BF16 rounding points within the
    trajectory tolerance, 1e-5 x extent (the weights are the network under
    test: both sides take the same values; the expected positions come from
    the oracle alone).
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, grid, make_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_trained_warm_start_beats_the_plain_step_at_one_iteration():
    from paper_2503_18616_gb300 import surrogate
    m = grid((9, 9, 5))
    p = inputs.default_params()
    tsim = make_sim([m], p, 256)
    tr = surrogate.train(tsim, [m], n_full=10, env_substeps=80_000, lr=1e-3, epochs=2, seed=3)
    tsim.close()
    assert tr["losses"][-1] < 0.5 * tr["losses"][0], tr["losses"]
    n_env, N, seed = 8, 40, 5
    envs = [0, 3, 7]
    om = oracle.Mesh(*m)
    V, ext = om.V, om.extent
    full = {}
    for e in envs:
        oe = oracle.Env(om, inputs.default_params(iterations=10))
        oe.reset(seed, e)
        oe.run(N, want_obs=False)
        full[e] = oe.state()[0]
    ws = make_sim([m], p, n_env, seed=seed)
    ws.set_network(tr["params"], *tr["norm"])
    for _ in range(N):
        ws.step_surrogate(float("inf"), 10)
    ws.sync()
    xw, _, _ = gpu_positions(ws)
    ps = make_sim([m], p, n_env, seed=seed)
    for _ in range(N):
        ps.step()
    ps.sync()
    xp, _, _ = gpu_positions(ps)
    err_w = max(np.abs(xw[e * V:(e + 1) * V] - full[e]).max() for e in envs) / ext
    err_p = max(np.abs(xp[e * V:(e + 1) * V] - full[e]).max() for e in envs) / ext
    print(f"after {N} steps vs the 10-iteration FP64 solve: warm-start {err_w:.3e}, "
          f"plain 1 iteration {err_p:.3e} x extent (ratio {err_w / err_p:.3f})")
    assert err_w <= 0.5 * err_p, (err_w, err_p)
    # the trained step is the oracle's surrogate step with the same weights
    net = oracle.Net.from_params(tr["params"], *tr["norm"], bf16=True)
    for e in envs:
        oe = oracle.Env(om, p)
        oe.reset(seed, e)
        for _ in range(N):
            oe.step_surrogate(net, np.inf, 10)
        assert np.abs(xw[e * V:(e + 1) * V] - oe.state()[0]).max() <= POS_TOL * ext, e
    ws.close()
    ps.close()
