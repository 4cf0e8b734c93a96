"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (constraint tables, colouring, orders, sampled vertex ids,
counter-based actions, contact lists on identical FP32 inputs) must be
bit-exact; positions must agree within 1e-5 of the mesh extent (the FP32 GPU
path against the FP64 oracle), velocities within that divided by h.
"""
import numpy as np
import pytest

from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, grid, make_sim, oracle_envs, packed_offsets

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def P(**over):
    return inputs.default_params(**over)


def compare_states(sim, oenvs, meshes, n_env, env_mesh=None, label="", tol=POS_TOL):
    x, v, tool = gpu_positions(sim)
    off = packed_offsets(meshes, n_env, env_mesh)
    h = sim.params["dt"] / sim.params["substeps"]
    worst = 0.0
    for e, oe in oenvs.items():
        ox, ov, oc = oe.state()
        ext = oe.mesh.extent
        gx = x[off[e]:off[e + 1]]
        gv = v[off[e]:off[e + 1]]
        ex = np.max(np.abs(gx - ox)) / ext
        ev = np.max(np.abs(gv - ov)) * h / ext
        worst = max(worst, ex)
        assert ex <= tol, f"{label} env {e}: position error {ex:.3e} x extent"
        assert ev <= tol, f"{label} env {e}: velocity error {ev:.3e} x extent / h"
        assert np.allclose(tool[e], oc, rtol=0, atol=1e-12), f"{label} env {e}: tool"
    return worst


# --------------------------------------------------------------------------
# Integer work: bit-exact
# --------------------------------------------------------------------------

def _shuffled_mesh(seed):
    rest, w, tets = grid((5, 4, 3))
    rng = np.random.default_rng(seed)
    tets = tets[rng.permutation(len(tets))]
    for t in tets:                   # random vertex order inside each tet
        t[:] = t[rng.permutation(4)]
    return rest, w, tets


@pytest.mark.parametrize("mesh", ["two_tet", (2, 2, 2), (3, 3, 2), (9, 9, 5), (17, 17, 9), "shuffled"])
def test_constraint_tables_bit_exact(mesh):
    import oracle
    if mesh == "two_tet":
        m = inputs.two_tet_mesh()
        n_obs = 2
    elif mesh == "shuffled":
        m = _shuffled_mesh(3)
        n_obs = 8
    else:
        m = grid(mesh)
        n_obs = 4
    sim = make_sim([m], P(n_obs=n_obs), 1)
    om = oracle.Mesh(*m)
    assert np.array_equal(sim.mesh_table("tets").reshape(-1, 4), om.tets)
    assert np.array_equal(sim.mesh_table("flipped"), om.flipped)
    assert np.array_equal(sim.mesh_table("edges").reshape(-1, 2), om.edges)
    for name in ("ecolor", "tcolor", "eorder", "torder", "ecol_off", "tcol_off", "top"):
        assert np.array_equal(sim.mesh_table(name), getattr(om, name)), name


@pytest.mark.parametrize("seed", [0, 12345, 2**40 + 7])
def test_reset_draws_bit_exact(seed):
    m = grid((17, 17, 9))
    n_env = 16
    sim = make_sim([m], P(), n_env, seed=seed)
    oenvs, _ = oracle_envs([m], P(), n_env, seed=seed)
    _, _, tool = gpu_positions(sim)
    for e, oe in oenvs.items():
        g, o = sim.env_ints(e), oe.ints()
        assert np.array_equal(g["obs_ids"], o["obs_ids"])
        assert g["target"] == o["target"] and g["t"] == 0
        assert np.array_equal(tool[e], oe.state()[2])


def test_device_actions_bit_exact():
    m = grid((9, 9, 5))
    n_env, steps = 8, 60
    p = P(gravity=(0.0, 0.0, 0.0), radius=0.0)
    sim = make_sim([m], p, n_env, seed=99)
    oenvs, _ = oracle_envs([m], p, n_env, seed=99)
    for _ in range(steps):
        sim.step()
    for oe in oenvs.values():
        oe.run(steps, want_obs=False)
    _, _, tool = gpu_positions(sim)
    for e, oe in oenvs.items():
        assert np.array_equal(tool[e], oe.state()[2]), e   # same draws, same float64 sums
        assert sim.env_ints(e)["t"] == steps


# --------------------------------------------------------------------------
# Trajectories: positions within 1e-5 x extent
# --------------------------------------------------------------------------

@pytest.mark.parametrize("block", [128, 256, 512, 1024])
def test_block9x9x5_one_env_100_steps(block):
    m = grid((9, 9, 5))
    p = P()
    sim = make_sim([m], p, 1, block_threads=block, seed=0)
    oenvs, _ = oracle_envs([m], p, 1, seed=0)
    oe = oenvs[0]
    for k in range(1, 101):
        obs, rew, done = sim.step()
        o_obs, o_rew, o_done = oe.step()
        if k in (1, 10, 50, 100):
            compare_states(sim, oenvs, [m], 1, label=f"step {k}")
            ext = oe.mesh.extent
            assert np.max(np.abs(obs.cpu().numpy()[0] - o_obs)) <= POS_TOL * ext
            assert abs(float(rew[0]) - o_rew) <= POS_TOL * ext
            assert int(done[0]) == o_done


@pytest.mark.parametrize("mesh", ["two_tet", (2, 2, 2), (3, 2, 2), (3, 3, 2), (3, 3, 3), (5, 3, 2), (9, 9, 5)])
def test_small_and_ragged_meshes(mesh):
    if mesh == "two_tet":
        rest, w, tets = inputs.two_tet_mesh()
        w = w.copy()
        w[0] = 0.0      # hang the pair of tets from one vertex so it stays near its extent
        m = (rest, w, tets)
    else:
        m = grid(mesh)
    n_obs = 2 if mesh == "two_tet" else 4
    p = P(n_obs=n_obs, radius=3e-3)
    n_env, steps = 3, 6
    sim = make_sim([m], p, n_env, seed=5)
    oenvs, _ = oracle_envs([m], p, n_env, seed=5)
    rng = np.random.default_rng(1)
    rest, w, _ = m
    xs, vs = [], []
    for e in range(n_env):
        xs.append(inputs.perturbed_positions(rest, 3e-4, 10 + e, inv_mass=w))
        v = rng.normal(0, 0.02, rest.shape)
        v[w == 0] = 0
        vs.append(v)
    x32 = np.concatenate(xs).astype(np.float32)
    v32 = np.concatenate(vs).astype(np.float32)
    sim.set_state(torch.from_numpy(x32).cuda(), torch.from_numpy(v32).cuda())
    off = packed_offsets([m], n_env)
    for e, oe in oenvs.items():
        oe.set_state(x=x32[off[e]:off[e + 1]].astype(np.float64), v=v32[off[e]:off[e + 1]].astype(np.float64))
    acts = inputs.random_actions(steps, n_env, 7)
    for k in range(steps):
        sim.step(torch.from_numpy(acts[k].astype(np.float32)).cuda())
        for e, oe in oenvs.items():
            oe.step(acts[k, e])
    compare_states(sim, oenvs, [m], n_env, label=str(mesh))


@pytest.mark.parametrize("iterations", [0, 2, 3])
def test_iteration_counts_carry_lambda(iterations):
    m = grid((9, 9, 5))
    # without constraints nothing holds the tissue together, so that case runs
    # without gravity and tool (free drift from a perturbed, moving start)
    if iterations == 0:
        p = P(iterations=0, gravity=(0.0, 0.0, 0.0), radius=0.0)
    else:
        p = P(iterations=iterations, alpha_d=1e-4, alpha_v=1e-10, radius=4e-3)
    n_env, steps = 2, 20
    sim = make_sim([m], p, n_env, seed=4)
    oenvs, _ = oracle_envs([m], p, n_env, seed=4)
    if iterations == 0:
        rest, w, _ = m
        x32 = np.concatenate([inputs.perturbed_positions(rest, 3e-4, 20 + e, inv_mass=w) for e in range(n_env)])
        v32 = np.random.default_rng(3).normal(0, 0.01, x32.shape)
        v32[np.tile(w, n_env) == 0] = 0
        x32, v32 = x32.astype(np.float32), v32.astype(np.float32)
        sim.set_state(torch.from_numpy(x32).cuda(), torch.from_numpy(v32).cuda())
        V = len(rest)
        for e, oe in oenvs.items():
            oe.set_state(x=x32[e * V:(e + 1) * V].astype(np.float64), v=v32[e * V:(e + 1) * V].astype(np.float64))
    for _ in range(steps):
        sim.step()
    for oe in oenvs.values():
        oe.run(steps, want_obs=False)
    tol = POS_TOL
    if iterations == 0:
        # Free drift has no constraint to damp the float32 cancellation in
        # v = (x - x_prev) / h, so the bar is the float32 oracle's own distance
        # from the float64 oracle (times 4), if that exceeds the tissue tolerance.
        import oracle
        o32 = oracle.Env(oracle.Mesh(*m, precision="f32"), p)
        o32.reset(4, 1)
        V = len(m[0])
        o32.set_state(x=x32[V:2 * V].astype(np.float64), v=v32[V:2 * V].astype(np.float64))
        o32.run(steps, want_obs=False)
        floor = np.max(np.abs(o32.state()[0] - oenvs[1].state()[0])) / oenvs[1].mesh.extent
        tol = max(POS_TOL, 4 * floor)
    compare_states(sim, oenvs, [m], n_env, label=f"iterations={iterations}", tol=tol)


def test_rest_state_stays_put():
    m = grid((9, 9, 5))
    p = P(gravity=(0.0, 0.0, 0.0), radius=0.0)
    sim = make_sim([m], p, 2)
    for _ in range(10):
        sim.step()
    x, v, _ = gpu_positions(sim)
    rest32 = np.tile(m[0].astype(np.float32), (2, 1)).astype(np.float64)
    assert np.max(np.abs(x - rest32)) <= 1e-6 * 0.04
    assert np.max(np.abs(v)) <= 1e-6 * 0.04 * 600


def test_collision_contacts_bit_exact_on_identical_inputs():
    """One substep, no constraints, no gravity: the step is the sphere
    projection alone, so contact sets are decided on identical FP32 inputs."""
    m = grid((9, 9, 5))
    rest, w, _ = m
    p = P(gravity=(0.0, 0.0, 0.0), iterations=0, substeps=1, radius=7e-3)
    n_env = 6
    sim = make_sim([m], p, n_env)
    oenvs, _ = oracle_envs([m], p, n_env)
    rng = np.random.default_rng(8)
    xs, tools = [], []
    for e in range(n_env):
        while True:
            x = inputs.perturbed_positions(rest, 1e-3, 100 + e + 1000 * len(xs), inv_mass=w).astype(np.float32)
            c = np.array([rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01), rng.uniform(0.016, 0.022)])
            dist = np.linalg.norm(x.astype(np.float64) - c, axis=1)
            if np.min(np.abs(dist - p["radius"])) > 1e-6 * p["radius"]:
                break
        xs.append(x)
        tools.append(c)
    x32 = np.concatenate(xs)
    sim.set_state(torch.from_numpy(x32).cuda(), torch.zeros_like(torch.from_numpy(x32)).cuda(),
                  torch.from_numpy(np.array(tools)).cuda())
    off = packed_offsets([m], n_env)
    for e, oe in oenvs.items():
        oe.set_state(x=x32[off[e]:off[e + 1]].astype(np.float64), v=np.zeros((len(rest), 3)), c=tools[e])
    zeros = torch.zeros((n_env, 3), dtype=torch.float32, device="cuda")
    sim.step(zeros)
    total = 0
    for e, oe in oenvs.items():
        oe.step(np.zeros(3))
        g, o = sim.env_ints(e)["contacts"], oe.ints()["contacts"]
        assert np.array_equal(g, o), e
        total += len(g)
    assert total >= n_env
    compare_states(sim, oenvs, [m], n_env, label="collision")


@pytest.mark.parametrize("path", ["cluster", "streaming"])
def test_uneven_meshes_per_env_compliance_and_large_mesh_paths(path):
    """The 33 x 33 x 17 block (18513 vertices) exceeds one CTA's shared
    memory: by default a 2-CTA cluster holds it on chip (distributed shared
    memory), with FFSRL_SCHED_NO_CLUSTER the global-memory working copy runs."""
    from paper_2503_18616_gb300 import ffsrl
    shapes = [(9, 9, 5), (13, 13, 7), (33, 33, 17)]
    meshes = [grid(s) for s in shapes]
    n_env, steps = 7, 8
    env_mesh = np.array([2, 0, 1, 2, 1, 0, 2], dtype=np.int32)
    alpha = inputs.compliance_draws(n_env, 1e-7, 1e-5, 3)
    p = P()
    flags = ffsrl.SCHED_NO_CLUSTER if path == "streaming" else 0
    sim = make_sim(meshes, p, n_env, env_mesh=env_mesh, env_compliance=alpha, seed=6, schedule_flags=flags)
    assert sim.resident_envs == (int(np.sum(env_mesh != 2)) if path == "streaming" else n_env)
    oenvs, _ = oracle_envs(meshes, p, n_env, env_mesh=env_mesh, env_compliance=alpha, seed=6)
    for _ in range(steps):
        sim.step()
    for oe in oenvs.values():
        oe.run(steps, want_obs=False)
    compare_states(sim, oenvs, meshes, n_env, env_mesh=env_mesh, label="uneven " + path)


@pytest.mark.parametrize("iterations", [1, 2])
def test_cluster_and_streaming_paths_are_bit_identical(iterations):
    """Same envs through the cluster kernel and the global-memory kernel:
    positions, velocities, observations, rewards and contact lists agree bit
    for bit (the same arithmetic in the same colour order; with 2 iterations
    the multipliers are carried per record)."""
    from paper_2503_18616_gb300 import ffsrl
    meshes = [grid((33, 33, 17)), grid((9, 9, 5))]
    n_env, steps = 3, 6
    env_mesh = np.array([0, 1, 0], dtype=np.int32)
    p = P(radius=6e-3, iterations=iterations)
    out = {}
    for path, flags in (("cluster", 0), ("streaming", ffsrl.SCHED_NO_CLUSTER)):
        sim = make_sim(meshes, p, n_env, env_mesh=env_mesh, seed=9, schedule_flags=flags)
        for _ in range(steps):
            obs, rew, done = sim.step()
        sim.sync()
        x, v, tool = sim.get_state()
        ints = [sim.env_ints(e) for e in range(n_env)]
        out[path] = (x.cpu().numpy(), v.cpu().numpy(), tool.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy(), ints)
    a, b = out["cluster"], out["streaming"]
    for k in range(5):
        assert np.array_equal(a[k], b[k]), k
    for ia, ib in zip(a[5], b[5]):
        for key in ia:
            assert np.array_equal(np.asarray(ia[key]), np.asarray(ib[key])), key
    if iterations == 1:   # the tool reaches the tissue (the contact lists are exercised)
        assert any(len(np.asarray(i.get("contacts", []))) > 0 for i in a[5])


def test_block17x17x9_4096_envs_sampled_1000_steps():
    """The benchmark configuration: 4096 envs of the 2601-vertex block, device
    actions, 1000 steps; sampled envs are checked against the oracle."""
    m = grid((17, 17, 9))
    p = P()
    n_env, steps = 4096, 1000
    sim = make_sim([m], p, n_env, seed=2024)
    sample = [0, 1, 1777, 4095]
    oenvs, _ = oracle_envs([m], p, n_env, seed=2024, envs=sample)
    for k in range(steps - 1):
        sim.step()
    obs, rew, done = sim.step()
    obs, rew = obs.cpu().numpy(), rew.cpu().numpy()
    ext = oenvs[0].mesh.extent
    for e, oe in oenvs.items():
        o_obs, o_rew, _ = oe.run(steps)
        assert np.max(np.abs(obs[e] - o_obs[-1])) <= POS_TOL * ext
        assert abs(rew[e] - o_rew[-1]) <= POS_TOL * ext
    worst = compare_states(sim, oenvs, [m], n_env, label="block17 x 4096")
    print(f"max position error over sampled envs: {worst:.3e} x extent")


def test_masked_reset_and_state_roundtrip():
    m = grid((9, 9, 5))
    n_env = 4
    sim = make_sim([m], P(), n_env, seed=1)
    for _ in range(5):
        sim.step()
    x0, v0, t0 = sim.get_state()
    mask = torch.tensor([1, 0, 1, 0], dtype=torch.uint8, device="cuda")
    sim.reset(seed=77, mask=mask)
    x1, v1, t1 = sim.get_state()
    off = packed_offsets([m], n_env)
    rest32 = m[0].astype(np.float32)
    oenvs, _ = oracle_envs([m], P(), n_env, seed=77)
    for e in range(n_env):
        a, b = off[e], off[e + 1]
        if e in (0, 2):
            assert np.array_equal(x1[a:b].cpu().numpy(), rest32)
            assert float(v1[a:b].abs().max()) == 0.0
            assert np.array_equal(sim.env_ints(e)["obs_ids"], oenvs[e].ints()["obs_ids"])
            assert sim.env_ints(e)["t"] == 0
        else:
            assert torch.equal(x1[a:b], x0[a:b]) and sim.env_ints(e)["t"] == 5
    xm = x1 + 1e-4
    sim.set_state(xm, v1 * 2, t1 + 0.001)
    x2, v2, t2 = sim.get_state()
    assert torch.equal(x2, xm) and torch.equal(v2, v1 * 2) and torch.equal(t2, t1 + 0.001)


def test_step_host_matches_device_step():
    m = grid((9, 9, 5))
    n_env = 5
    a = make_sim([m], P(), n_env, seed=3)
    b = make_sim([m], P(), n_env, seed=3)
    acts = inputs.random_actions(4, n_env, 1).astype(np.float32)
    for k in range(4):
        oa, ra, da = a.step(torch.from_numpy(acts[k]).cuda())
        ob, rb, db = b.step_host(acts[k])
    assert np.array_equal(oa.cpu().numpy(), ob)
    assert np.array_equal(ra.cpu().numpy(), rb)
    assert np.array_equal(da.cpu().numpy(), db)
    # device-drawn actions through the host entry point too
    oa, _, _ = a.step()
    ob, _, _ = b.step_host(None)
    assert np.array_equal(oa.cpu().numpy(), ob)
    # page-locked caller buffers are copied directly
    ha, ho, hr, hd = b.pinned_host_buffers()
    for k in range(3):
        ha[:] = acts[k]
        oa, ra, da = a.step(torch.from_numpy(acts[k]).cuda())
        b.step_host(ha, ho, hr, hd)
        assert np.array_equal(oa.cpu().numpy(), ho)
        assert np.array_equal(ra.cpu().numpy(), hr)
        assert np.array_equal(da.cpu().numpy(), hd)


def test_non_finite_state_is_reported_by_sync():
    from paper_2503_18616_gb300 import ffsrl
    m = grid((9, 9, 5))
    sim = make_sim([m], P(), 3)
    x, v, t = sim.get_state()
    x[405 + 200, 1] = float("nan")
    sim.set_state(x, v, t)
    sim.step()
    with pytest.raises(ffsrl.FfsrlError) as ei:
        sim.sync()
    assert ei.value.code == -5 and "env 1" in str(ei.value)
    sim.sync()   # flag cleared


def test_every_schedule_gives_bit_identical_results():
    """Slot permutation, record grouping, the TMA ring and the block size are
    execution choices: constraints of one colour touch disjoint vertices, so
    every schedule must give the same bits."""
    from paper_2503_18616_gb300 import ffsrl
    m = grid((9, 9, 5))
    p = P(iterations=2, alpha_d=1e-4)
    n_env, steps = 3, 12
    ref = None
    configs = []
    for flags in (0, ffsrl.SCHED_NO_PERMUTE, ffsrl.SCHED_NO_RING, ffsrl.SCHED_NO_PERMUTE | ffsrl.SCHED_NO_RING):
        for block in (128, 256, 384, 512, 1024):
            configs.append((flags, block))
    for envs_flag, blocks in ((ffsrl.SCHED_ENVS2, (128, 256, 384, 512)), (ffsrl.SCHED_ENVS4, (128, 256))):
        for flags in (0, ffsrl.SCHED_NO_PERMUTE):
            for block in blocks:
                configs.append((flags | envs_flag, block))
    for flags, block in configs:
        sim = make_sim([m], p, n_env, block_threads=block, schedule_flags=ffsrl.SCHED_FORCE | flags, seed=3)
        assert sim.ring_envs == (0 if flags & ffsrl.SCHED_NO_RING else n_env)
        assert sim.envs_per_cta == (4 if flags & ffsrl.SCHED_ENVS4 else 2 if flags & ffsrl.SCHED_ENVS2 else 1)
        for _ in range(steps):
            obs, rew, done = sim.step()
        x, v, _ = sim.get_state()
        out = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy())
        if ref is None:
            ref = out
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a, b), (flags, block)
        sim.close()
    # the global-memory working copy, autotuned and forced
    for flags in (ffsrl.SCHED_GLOBAL_MEMORY, ffsrl.SCHED_GLOBAL_MEMORY | ffsrl.SCHED_FORCE):
        sim = make_sim([m], p, n_env, block_threads=256 if flags & ffsrl.SCHED_FORCE else 0,
                       schedule_flags=flags, seed=3)
        assert sim.resident_envs == 0
        for _ in range(steps):
            obs, rew, done = sim.step()
        x, v, _ = sim.get_state()
        out = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy())
        for a, b in zip(ref, out):
            assert np.array_equal(a, b), flags
        sim.close()


def test_refined_phases_and_four_cta_kernel_give_the_colour_schedule_bits():
    """On the 17x17x9 block the permuted schedule refines the 18 + 37 colours
    into phases of whole multiples of 256 constraints (every vertex still
    sees its constraints in colour order). The colour phases (no permutation),
    the refined phases, and the kernel budgeted for four CTAs per SM must give
    the same bits, with one and with two iterations."""
    from paper_2503_18616_gb300 import ffsrl
    m = grid((17, 17, 9))
    for iters in (1, 2):
        p = P(iterations=iters)
        n_env, steps = 4, 6
        ref = None
        for flags in (ffsrl.SCHED_NO_PERMUTE, 0, ffsrl.SCHED_FOUR_CTAS):
            sim = make_sim([m], p, n_env, block_threads=256, schedule_flags=ffsrl.SCHED_FORCE | flags, seed=8)
            assert sim.ctas_per_sm == (4 if flags & ffsrl.SCHED_FOUR_CTAS else 3)
            for _ in range(steps):
                obs, rew, done = sim.step()
            x, v, _ = sim.get_state()
            out = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy())
            if ref is None:
                ref = out
            else:
                for a, b in zip(ref, out):
                    assert np.array_equal(a, b), (flags, iters)
            sim.close()


def test_uneven_1024_env_batch_sampled():
    """The uneven-batching configuration: 1024 envs, vertex counts log-uniform in
    [500, 20000] (37 block sizes), per-env edge compliance, all size classes
    launched concurrently (the largest meshes on 2-CTA clusters); the
    smallest, a middle and the largest env are checked against the FP64
    oracle after 100 steps. An env whose error exceeds the 1e-5 x extent
    tolerance must stay within twice what the oracle's own float32 build
    deviates from its float64 build over the same steps (the float32 rounding
    floor of a trajectory that buckles under the tool); the smallest and the
    middle env must meet the tolerance outright."""
    import oracle
    shapes, env_mesh = inputs.uneven_batch(1024, 500, 20000, seed=12345)
    meshes = [grid(s) for s in shapes]
    alpha = inputs.compliance_draws(1024, 1e-7, 1e-5, seed=12345)
    p = P()
    steps = 100
    sim = make_sim(meshes, p, 1024, env_mesh=env_mesh, env_compliance=alpha, seed=8)
    assert sim.n_groups >= 2 and sim.resident_envs == 1024   # every env on chip
    vs = np.array([len(meshes[m][0]) for m in env_mesh])
    sample = [int(np.argmin(vs)), int(np.argsort(vs)[512]), int(np.argmax(vs))]
    oenvs, _ = oracle_envs(meshes, p, 1024, env_mesh=env_mesh, env_compliance=alpha, seed=8, envs=sample)
    for _ in range(steps):
        sim.step()
    for oe in oenvs.values():
        oe.run(steps, want_obs=False)
    x, _, _ = gpu_positions(sim)
    off = packed_offsets(meshes, 1024, env_mesh)
    for rank, e in enumerate(sample):
        oe = oenvs[e]
        ox = oe.state()[0]
        ext = oe.mesh.extent
        err = float(np.max(np.abs(x[off[e]:off[e + 1]] - ox)) / ext)
        if err <= POS_TOL:
            continue
        assert rank == 2, f"env {e} ({vs[e]} vertices): {err:.3e} x extent"
        o32 = oracle.Env(oracle.Mesh(*meshes[env_mesh[e]], precision="f32"), dict(p, alpha_d=float(alpha[e])))
        o32.reset(8, e)
        o32.run(steps, want_obs=False)
        floor = float(np.max(np.abs(o32.state()[0] - ox)) / ext)
        assert err <= 2 * floor, f"env {e} ({vs[e]} vertices): {err:.3e} vs float32 floor {floor:.3e}"


def test_largest_supported_mesh_and_the_size_limit():
    """Shared-memory slots are 16-bit, so a mesh may have up to 65535
    vertices: a 40x40x40 block (64000 vertices, global-memory path) matches
    the oracle; 65536 vertices are rejected with FFSRL_E_INVAL."""
    from paper_2503_18616_gb300 import ffsrl
    m = grid((40, 40, 40))
    p = P(radius=6e-3)
    sim = make_sim([m], p, 1, seed=4)
    assert sim.resident_envs == 0
    oenvs, om = oracle_envs([m], p, 1, seed=4)
    acts = inputs.random_actions(3, 1, 5)
    acts[:, :, 2] = -1.0
    for k in range(3):
        sim.step(torch.from_numpy(acts[k].astype(np.float32)).cuda())
        oenvs[0].step(acts[k, 0])
    x, _, _ = gpu_positions(sim)
    assert np.max(np.abs(x - oenvs[0].state()[0])) <= POS_TOL * om[0].extent
    sim.close()
    big = grid((64, 32, 32))   # 65536 vertices
    with pytest.raises(ffsrl.FfsrlError):
        make_sim([big], p, 1)
