"""Tissue connections (Sec. III-A) on the GPU against the oracle (pinned in
test_oracle_connection_pins.py): a tissue block connected to the base block
beneath it.

Connection tables and objects are integer work and must be bit-exact;
trajectories (sphere tool, random actions; one and two iterations; the
grasper lifting the connected tissue) are held to 1e-5 x extent; every execution schedule must give the same bits.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, packed_offsets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

R = 6e-3   # connection radius: the tissue's bottom layer, 1 mm above the base


def _sim(mesh, p, n_env, seed=0, **kw):
    from paper_2503_18616_gb300 import build, ffsrl
    build.build()
    sim = ffsrl.Sim([mesh], p, n_env, **kw)
    sim.reset(seed)
    return sim


def _oracle(mesh, p, n_env, seed=0):
    om = oracle.Mesh(*mesh, conn_radius=p["conn_radius"])
    envs = {}
    for e in range(n_env):
        envs[e] = oracle.Env(om, p)
        envs[e].reset(seed, e)
    return envs, om


@pytest.mark.parametrize("shape,gap,radius", [((3, 3, 2, 2), 1e-3, 5e-3), ((5, 4, 2, 3), 0.0, 4e-3),
                                              ((17, 17, 5, 5), 1e-3, R)])
def test_connection_tables_bit_exact(shape, gap, radius):
    mesh = inputs.stacked_blocks(*shape, gap=gap)
    sim = _sim(mesh, inputs.default_params(conn_radius=radius, n_obs=4), 1)
    om = oracle.Mesh(*mesh, conn_radius=radius)
    assert om.C > 0
    assert np.array_equal(sim.mesh_table("conns").reshape(-1, 4), om.conns)
    assert np.array_equal(sim.mesh_table("corder"), om.corder)
    assert np.array_equal(sim.mesh_table("ccol_off"), om.ccol_off)
    assert np.array_equal(sim.mesh_table("objects"), om.objects)
    sim.close()


def _actions(steps, n_env, seed):
    a = inputs.random_actions(steps, n_env, seed)
    a[: steps // 3, :, 2] = -1.0    # press into the tissue first
    return a


@pytest.mark.parametrize("shape,n_env,steps,iters", [((9, 9, 3, 3), 3, 40, 1), ((9, 9, 3, 3), 2, 30, 2),
                                                     ((17, 17, 5, 5), 2, 20, 1)])
def test_connected_tissue_trajectories_match_oracle(shape, n_env, steps, iters):
    mesh = inputs.stacked_blocks(*shape, gap=1e-3)
    p = inputs.default_params(conn_radius=R, iterations=iters)
    sim = _sim(mesh, p, n_env, seed=4)
    oenvs, om = _oracle(mesh, p, n_env, seed=4)
    acts = _actions(steps, n_env, 9)
    for k in range(steps):
        obs, rew, done = sim.step(torch.from_numpy(acts[k].astype(np.float32)).cuda())
        for e, oe in oenvs.items():
            oo, orw, od = oe.step(acts[k, e])
    x, v, tool = gpu_positions(sim)
    off = packed_offsets([mesh], n_env)
    h = p["dt"] / p["substeps"]
    tol = POS_TOL * om.extent
    nb = shape[0] * shape[1] * shape[2]
    for e, oe in oenvs.items():
        ox, ov, oc = oe.state()
        assert np.max(np.abs(x[off[e]:off[e + 1]] - ox)) <= tol, e
        assert np.max(np.abs(v[off[e]:off[e + 1]] - ov)) * h <= tol, e
        assert np.array_equal(tool[e], oc)
        # the tissue moved (sagged onto its connections and was pressed)
        assert np.max(np.abs(ox[nb:] - mesh[0][nb:])) > 1e-4
    sim.close()


def test_grasper_lifts_the_connected_tissue_like_the_oracle():
    """The retraction task: closed clamps grasp the tissue's top centre and
    lift; the connections hold its bottom to the base."""
    mesh = inputs.stacked_blocks(9, 9, 3, 3, gap=1e-3)
    p = inputs.default_params(conn_radius=R, tool_model=1, grasp_radius=3e-3, iterations=2)
    n_env = 2
    sim = _sim(mesh, p, n_env, seed=2)
    oenvs, om = _oracle(mesh, p, n_env, seed=2)
    top = float(mesh[0][:, 2].max())
    c = np.array([[0.0, 0.0, top + p["clamp_length"] + 0.4e-3], [5e-3, 5e-3, top + p["clamp_length"] + 0.4e-3]])
    ang = float(np.float32(math.radians(1.0)))
    sim.set_state(tool=torch.from_numpy(c).cuda())
    sim.set_clamp_angles(torch.full((n_env,), ang, dtype=torch.float32).cuda())
    for e, oe in oenvs.items():
        oe.set_state(c=c[e])
        oe.set_clamp(ang)
    acts = [np.zeros(3)] + [np.array([0.0, 0.0, 1.0])] * 6
    for a in acts:
        sim.step(torch.from_numpy(np.tile(a, (n_env, 1)).astype(np.float32)).cuda())
        for oe in oenvs.values():
            oe.step(a)
        g = sim.grasp()
        assert [int(v) for v in g] == [oenvs[e].ints()["grasp"] for e in range(n_env)]
    assert (g >= 0).all()
    x, _, _ = gpu_positions(sim)
    off = packed_offsets([mesh], n_env)
    # contact decisions amplify rounding: the bar is 1e-5 x extent or four
    # times the distance between the oracle's FP32 and FP64 builds
    om32 = oracle.Mesh(*mesh, conn_radius=R, precision="f32")
    nb = 9 * 9 * 3
    for e, oe in oenvs.items():
        o32 = oracle.Env(om32, p)
        o32.reset(2, e)
        o32.set_state(c=c[e])
        o32.set_clamp(ang)
        for a in acts:
            o32.step(a)
        ox = oe.state()[0]
        floor = np.max(np.abs(o32.state()[0] - ox))
        tol = max(POS_TOL * om.extent, 4 * floor)
        assert np.max(np.abs(x[off[e]:off[e + 1]] - ox)) <= tol, (e, floor / om.extent)
        xe = x[off[e]:off[e + 1]]
        assert xe[g[e], 2] > top + 5e-3                       # the grasped vertex went up
        assert np.max(np.abs(xe[nb:nb + 81, 2] - mesh[0][nb:nb + 81, 2])) < 3e-3   # the bottom stays attached
    sim.close()


def test_connections_every_schedule_gives_bit_identical_results():
    from paper_2503_18616_gb300 import ffsrl
    mesh = inputs.stacked_blocks(9, 9, 3, 3, gap=1e-3)
    p = inputs.default_params(conn_radius=R, iterations=2)
    n_env, steps = 4, 10
    acts = torch.from_numpy(_actions(steps, n_env, 5).astype(np.float32)).cuda()
    ref = None
    for flags, block in ((0, 256), (ffsrl.SCHED_NO_PERMUTE, 256), (ffsrl.SCHED_NO_RING, 512),
                         (ffsrl.SCHED_ENVS2, 128), (ffsrl.SCHED_ENVS4, 256)):
        sim = _sim(mesh, p, n_env, seed=5, block_threads=block, schedule_flags=ffsrl.SCHED_FORCE | flags)
        for k in range(steps):
            obs, rew, done = sim.step(acts[k])
        x, v, _ = sim.get_state()
        out = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy())
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), (flags, block)
        sim.close()


def test_connections_refuse_jacobi_and_warm_start():
    from paper_2503_18616_gb300 import ffsrl
    mesh = inputs.stacked_blocks(5, 5, 2, 2, gap=1e-3)
    with pytest.raises(ffsrl.FfsrlError):
        _sim(mesh, inputs.default_params(conn_radius=R, solver=1, n_obs=4), 1)
    _sim(mesh, inputs.default_params(solver=1, n_obs=4), 1).close()   # without connections: accepted
    sim = _sim(mesh, inputs.default_params(conn_radius=R, n_obs=4), 2)
    with pytest.raises(ffsrl.FfsrlError):
        sim.record_step(10)
    sim.close()


def test_large_connected_mesh_takes_the_global_memory_path():
    """19602 vertices exceed one CTA's shared memory; meshes with connections
    skip the cluster kernel, so this runs the global-memory variant."""
    mesh = inputs.stacked_blocks(33, 33, 9, 9, gap=1e-3)
    p = inputs.default_params(conn_radius=R, radius=6e-3)
    n_env, steps = 2, 6
    sim = _sim(mesh, p, n_env, seed=1)
    oenvs, om = _oracle(mesh, p, n_env, seed=1)
    assert om.C > 0
    acts = _actions(steps, n_env, 2)
    for k in range(steps):
        sim.step(torch.from_numpy(acts[k].astype(np.float32)).cuda())
        for e, oe in oenvs.items():
            oe.step(acts[k, e])
    x, _, _ = gpu_positions(sim)
    off = packed_offsets([mesh], n_env)
    for e, oe in oenvs.items():
        assert np.max(np.abs(x[off[e]:off[e + 1]] - oe.state()[0])) <= POS_TOL * om.extent, e
    sim.close()
