"""The paper's grasper tool (three capsules through a remote centre of
motion, against the surface faces) on the GPU, against the oracle (pinned in
test_oracle_grasper_pins.py).

Face tables are integer work and must be bit-exact; positions are held to
the trajectory tolerance (or, where contact decisions amplify rounding, to
four times the distance between the oracle's FP32 and FP64 builds); every
execution schedule must give the same bits.
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, grid, make_sim, oracle_envs, packed_offsets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def P(**over):
    return inputs.default_params(tool_model=1, **over)


@pytest.mark.parametrize("shape", [(3, 3, 2), (9, 9, 5), (17, 17, 9)])
def test_face_tables_bit_exact(shape):
    m = grid(shape)
    sim = make_sim([m], P(n_obs=4), 1)
    om = oracle.Mesh(*m)
    assert np.array_equal(sim.mesh_table("faces").reshape(-1, 3), om.faces)
    assert np.array_equal(sim.mesh_table("face_opposite"), om.face_opposite)
    assert np.array_equal(sim.mesh_table("forder"), om.forder)
    assert np.array_equal(sim.mesh_table("fcol_off"), om.fcol_off)


def _actions(steps, n_env, seed):
    """Down into the tissue for the first third, then a seeded random walk."""
    a = inputs.random_actions(steps, n_env, seed)
    a[: steps // 3, :, 2] = -1.0
    return a


@pytest.mark.parametrize("shape,n_env,steps", [((9, 9, 5), 3, 24), ((17, 17, 9), 2, 18)])
def test_grasper_trajectories_match_oracle(shape, n_env, steps):
    m = grid(shape)
    p = P()
    sim = make_sim([m], p, n_env, seed=7)
    oenvs, om = oracle_envs([m], p, n_env, seed=7)
    acts = _actions(steps, n_env, 3)
    contacts_seen = 0
    o_rew = {}
    for k in range(steps):
        obs, rew, done = sim.step(torch.from_numpy(acts[k].astype(np.float32)).cuda())
        for e, oe in oenvs.items():
            _, o_rew[e], _ = oe.step(acts[k, e])
    x, v, tool = gpu_positions(sim)
    off = packed_offsets([m], n_env)
    h = p["dt"] / p["substeps"]
    ext = om[0].extent
    # contact decisions make the grasper's trajectories sensitive to rounding:
    # the bar is 1e-5 x extent or, if larger, four times the
    # distance between the oracle's own FP32 and FP64 builds
    om32 = oracle.Mesh(*m, precision="f32")
    for e, oe in oenvs.items():
        ox, ov, oc = oe.state()
        o32 = oracle.Env(om32, p)
        o32.reset(7, e)
        for k in range(steps):
            o32.step(acts[k, e])
        floor = np.max(np.abs(o32.state()[0] - ox))
        tol = max(POS_TOL * ext, 4 * floor)
        assert np.max(np.abs(x[off[e]:off[e + 1]] - ox)) <= tol, (e, floor / ext)
        assert np.max(np.abs(v[off[e]:off[e + 1]] - ov)) * h <= tol, e
        assert np.array_equal(tool[e], oc)
        g, o = sim.env_ints(e)["contacts"], oe.ints()["contacts"]
        contacts_seen += len(o)
        assert len(set(g.tolist()) ^ set(o.tolist())) <= 2, (e, g, o)   # at most a boundary vertex each way
        assert abs(float(rew[e]) - o_rew[e]) <= tol
    assert contacts_seen > 0


def test_grasper_every_schedule_gives_bit_identical_results():
    from paper_2503_18616_gb300 import ffsrl
    m = grid((9, 9, 5))
    p = P(iterations=2)
    n_env, steps = 4, 10
    acts = torch.from_numpy(_actions(steps, n_env, 5).astype(np.float32)).cuda()
    ref = None
    for flags, block in ((0, 256), (ffsrl.SCHED_NO_PERMUTE, 256), (ffsrl.SCHED_NO_RING, 512),
                         (ffsrl.SCHED_ENVS2, 128), (ffsrl.SCHED_ENVS4, 256)):
        sim = make_sim([m], p, n_env, block_threads=block, schedule_flags=ffsrl.SCHED_FORCE | flags, seed=5)
        for k in range(steps):
            obs, rew, done = sim.step(acts[k])
        x, v, _ = sim.get_state()
        out = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy(),
               [sim.env_ints(e)["contacts"] for e in range(n_env)])
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref[:4], out[:4]):
                assert np.array_equal(a, b), (flags, block)
            for a, b in zip(ref[4], out[4]):
                assert np.array_equal(a, b), (flags, block)
        sim.close()


def test_dragging_matches_oracle():
    """Dragging constraint (Sec. III-A): four envs of a 9x9x5 block with the
    tool placed over the top face; env 0 and 1 close their clamps within reach
    of a vertex (grasped, then lifted), env 2 keeps them open, env 3 closes
    them out of reach. Grasped ids must equal the oracle's; positions follow
    the trajectory bar; opening the clamps releases."""
    import math
    m = grid((9, 9, 5))
    p = P(grasp_radius=3e-3)
    n_env = 4
    sim = make_sim([m], p, n_env, seed=2)
    oenvs, om = oracle_envs([m], p, n_env, seed=2)
    top = float(m[0][:, 2].max())
    L = p["clamp_length"]
    c = np.array([[0.0, 0.0, top + L + 0.4e-3], [3.5e-3, -1.0e-3, top + L + 0.4e-3],
                  [0.0, 0.0, top + L + 0.4e-3], [0.0, 0.0, top + L + 6e-3]])
    angles = np.array([math.radians(1.0), math.radians(1.0), math.radians(10.0), math.radians(1.0)])
    sim.set_state(tool=torch.from_numpy(c).cuda())
    sim.set_clamp_angles(torch.from_numpy(angles.astype(np.float32)).cuda())
    for e, oe in oenvs.items():
        oe.set_state(c=c[e])
        oe.set_clamp(float(np.float32(angles[e])))
    om32 = oracle.Mesh(*m, precision="f32")
    o32 = {}
    for e in range(n_env):
        o32[e] = oracle.Env(om32, p)
        o32[e].reset(2, e)
        o32[e].set_state(c=c[e])
        o32[e].set_clamp(float(np.float32(angles[e])))
    acts = [np.zeros(3)] + [np.array([0.0, 0.0, 1.0])] * 5
    for a in acts:
        sim.step(torch.from_numpy(np.tile(a, (n_env, 1)).astype(np.float32)).cuda())
        for e in range(n_env):
            oenvs[e].step(a)
            o32[e].step(a)
        g = sim.grasp()
        assert [int(x) for x in g] == [oenvs[e].ints()["grasp"] for e in range(n_env)]
    assert g[0] >= 0 and g[1] >= 0 and g[0] != g[1] and g[2] == -1 and g[3] == -1
    x, v, tool = gpu_positions(sim)
    off = packed_offsets([m], n_env)
    ext = om[0].extent
    for e in range(n_env):
        ox = oenvs[e].state()[0]
        floor = np.max(np.abs(o32[e].state()[0] - ox))
        tol = max(POS_TOL * ext, 4 * floor)
        assert np.max(np.abs(x[off[e]:off[e + 1]] - ox)) <= tol, (e, floor / ext)
    for e in (0, 1):   # the grasped vertex went up with the tool
        assert x[off[e] + g[e], 2] > top + 5e-3
    sim.set_clamp_angles(torch.full((n_env,), math.radians(10.0), dtype=torch.float32).cuda())
    sim.step(torch.zeros((n_env, 3), dtype=torch.float32).cuda())
    assert (sim.grasp() == -1).all()
    sim.close()
