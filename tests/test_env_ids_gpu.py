"""Global env ids of the counter-based draws (ffsrl_set_env_ids).

A shard of a batch, given the global ids of its envs, must draw for them what
the one-process run draws (Sec. III-B: envs are independent slices of one
batch): the observed vertices and the target vertex bit for bit, the device
actions bit for bit (tool positions), and the trajectories within the
position tolerance, against the FP64 oracle reset with the same global ids.
"""
import numpy as np
import pytest

from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, grid, make_sim, oracle_envs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.mark.parametrize("auto_reset", [0, 1])
def test_shard_with_global_ids_draws_as_the_whole_batch(auto_reset):
    m = grid((9, 9, 5))
    p = inputs.default_params(radius=4e-3, auto_reset=auto_reset, max_steps=4 if auto_reset else 0)
    ids = [5, 2, 9, 2]          # any ids, repeats allowed
    seed, steps = 13, 9
    sim = make_sim([m], p, len(ids), seed=seed)
    sim.set_env_ids(ids)
    sim.reset(seed)
    for _ in range(steps):
        obs, rew, _ = sim.step()
    sim.sync()
    x, _, tool = gpu_positions(sim)
    oenvs, om = oracle_envs([m], p, 10, seed=seed, envs=sorted(set(ids)))
    o_last = {}
    for g, oe in oenvs.items():
        for _ in range(steps):
            o_last[g] = oe.step()
    V, ext = om[0].V, om[0].extent
    for e, g in enumerate(ids):
        oe = oenvs[g]
        ints = sim.env_ints(e)
        oi = oe.ints()
        assert np.array_equal(ints["obs_ids"], oi["obs_ids"]) and ints["target"] == oi["target"], e
        assert np.array_equal(tool[e], oe.state()[2]), e
        assert np.max(np.abs(x[e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext, e
        assert abs(float(rew[e]) - o_last[g][1]) <= POS_TOL * ext
    # envs 1 and 3 share id 2: the same episode, bit for bit
    assert np.array_equal(x[V:2 * V], x[3 * V:4 * V])
    # back to the default ids: env e draws as id e again
    sim.set_env_ids(None)
    sim.reset(seed)
    sim.step()
    sim.sync()
    oe0, _ = oracle_envs([m], p, 1, seed=seed, envs=[1])
    assert np.array_equal(sim.env_ints(1)["obs_ids"], oe0[1].ints()["obs_ids"])
    sim.close()
