"""The allocation-free step entry point (ffsrl_step_noalloc).

It exists for callers that must not call cudaMalloc or cudaFree while they
step the simulation (real-time loops, where those calls can stall the device;
processes whose device memory is reserved up front by another allocator;
plugin hosts that forbid allocation per step). Its scratch is a fixed static
device array, so this test checks, through the C ABI, that two calls in a row
give the same states as the ordinary ffsrl_step on the same inputs, and that a
simulator too large for the static array is refused with a clear message.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, grid, make_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.mark.parametrize("iterations", [1, 3])
def test_noalloc_step_matches_ffsrl_step_twice(iterations):
    m = grid((9, 9, 5))
    p = inputs.default_params(iterations=iterations, alpha_d=1e-4, radius=4e-3)
    n_env = 5
    sim = make_sim([m], p, n_env, seed=9)
    rest, w, _ = m
    x0 = np.concatenate([inputs.perturbed_positions(rest, 3e-4, 40 + e, inv_mass=w) for e in range(n_env)])
    x0 = torch.from_numpy(x0.astype(np.float32)).cuda()
    v0 = torch.zeros_like(x0)
    _, _, tool0 = sim.get_state()
    sim.set_state(x0, v0, tool0)
    # the caller's own buffers, advanced without allocation
    x, v, tool = x0.clone(), v0.clone(), tool0.clone()
    acts = inputs.random_actions(2, n_env, 5).astype(np.float32)
    ext = 0.04
    for k in range(2):
        a = torch.from_numpy(acts[k]).cuda()
        sim.step_noalloc(a, x, v, tool)
        sim.step(a)
        xs, vs, ts = sim.get_state()
        torch.cuda.synchronize()
        h = p["dt"] / p["substeps"]
        assert float((x - xs).abs().max()) <= POS_TOL * ext, k
        assert float((v - vs).abs().max()) * h <= POS_TOL * ext, k
        assert float((tool - ts).abs().max()) <= 1e-12, k
        assert not torch.equal(x, x0)   # the state did move
    sim.close()


def test_noalloc_step_rejects_a_sim_beyond_the_scratch_size():
    from paper_2503_18616_gb300 import ffsrl
    m = grid((17, 17, 9))
    n_env = 512   # 512 x 2624 padded rows x 36 B > 32 MiB
    sim = make_sim([m], inputs.default_params(), n_env)
    x, v, tool = sim.get_state()
    a = torch.zeros((n_env, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ffsrl.FfsrlError) as ei:
        sim.step_noalloc(a, x, v, tool)
    assert ei.value.code == -1
    assert "scratch" in str(ei.value) and str(ffsrl.NOALLOC_SCRATCH_BYTES) in str(ei.value)
    sim.close()
