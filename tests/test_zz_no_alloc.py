"""The allocation-free step entry point (ffsrl_step_noalloc).

It exists for callers that must not call cudaMalloc or cudaFree while they
step the simulation (real-time loops, where those calls can stall the device;
processes whose device memory is reserved up front by another allocator;
plugin hosts that forbid allocation per step). Its scratch is a fixed static
device array, so this test checks, through the C ABI, that two calls in a row
give bit for bit the states of the ordinary ffsrl_step on the same inputs
(the two run the same kernels and schedule), on a resident single-group sim,
an uneven sim of several launch groups, a mesh held by a thread-block
cluster and the same mesh on the global-memory working copy; that the
device's free memory does not change across the calls; that ffsrl_sync
reports no error afterwards; and that a simulator too large for the static
array, or one with the grasper tool, is refused with a clear message.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2503_18616_gb300 import inputs
from sim_helpers import grid, make_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _run_pair(meshes, p, n_env, env_mesh=None, schedule_flags=0, seed=9):
    """Steps the same perturbed state twice with ffsrl_step_noalloc (caller
    buffers) and ffsrl_step (the sim's own state) and asserts equal bits."""
    sim = make_sim(meshes, p, n_env, env_mesh=env_mesh, seed=seed, schedule_flags=schedule_flags)
    parts = []
    for e in range(n_env):
        rest, w, _ = meshes[0 if env_mesh is None else int(env_mesh[e])]
        parts.append(inputs.perturbed_positions(rest, 3e-4, 40 + e, inv_mass=w))
    x0 = torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda()
    v0 = torch.zeros_like(x0)
    _, _, tool0 = sim.get_state()
    sim.set_state(x0, v0, tool0)
    x, v, tool = x0.clone(), v0.clone(), tool0.clone()
    acts = inputs.random_actions(2, n_env, 5).astype(np.float32)
    free = []
    for k in range(2):
        a = torch.from_numpy(acts[k]).cuda()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        sim.step_noalloc(a, x, v, tool)
        torch.cuda.synchronize()
        free.append((free_before, torch.cuda.mem_get_info()[0]))
        sim.step(a)
        xs, vs, ts = sim.get_state()
        torch.cuda.synchronize()
        assert torch.equal(x, xs), k
        assert torch.equal(v, vs), k
        assert torch.equal(tool, ts), k
        assert not torch.equal(x, x0)   # the state did move
    sim.sync()   # no device error was recorded by either call
    # the second call (after the first has looked up the scratch address)
    # leaves the device's free memory as it found it
    assert free[1][0] == free[1][1], free
    sim.close()


@pytest.mark.parametrize("iterations", [1, 3])
def test_noalloc_step_equals_ffsrl_step_twice(iterations):
    p = inputs.default_params(iterations=iterations, alpha_d=1e-4, radius=4e-3)
    _run_pair([grid((9, 9, 5))], p, 5)


def test_noalloc_step_on_an_uneven_batch_of_several_launch_groups():
    meshes = [grid((9, 9, 5)), grid((17, 17, 9)), grid((5, 5, 3))]
    env_mesh = np.array([0, 1, 2, 1, 0, 2], np.int32)
    p = inputs.default_params(alpha_d=1e-4, radius=4e-3, n_obs=4)
    _run_pair(meshes, p, len(env_mesh), env_mesh=env_mesh)


@pytest.mark.parametrize("path", ["cluster", "global"])
def test_noalloc_step_on_a_mesh_beyond_one_cta(path):
    """A 31 x 31 x 16 block (15376 vertices) is too large for one CTA's shared
    memory: it runs on a thread-block cluster, or with FFSRL_SCHED_NO_CLUSTER
    on the global-memory working copy that the scratch array also holds."""
    from paper_2503_18616_gb300 import ffsrl
    flags = ffsrl.SCHED_NO_CLUSTER if path == "global" else 0
    p = inputs.default_params(alpha_d=1e-4, radius=4e-3)
    _run_pair([grid((31, 31, 16))], p, 2, schedule_flags=flags)


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


def test_noalloc_step_rejects_the_grasper():
    from paper_2503_18616_gb300 import ffsrl
    sim = make_sim([grid((9, 9, 5))], inputs.default_params(tool_model=1), 2)
    x, v, tool = sim.get_state()
    a = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ffsrl.FfsrlError) as ei:
        sim.step_noalloc(a, x, v, tool)
    assert ei.value.code == -1 and "grasp" in str(ei.value)
    sim.close()
