"""Surrogate-assisted substeps on the GPU against the oracle.

Features and recorded training targets of the GPU pipeline must match the
oracle's within float32 rounding of positions (1e-5 x extent for targets
measured in position units, and the same relative bar for velocity-based
features); whole surrogate steps must match the oracle's surrogate step
within the trajectory tolerance, including the limiting cases (zero network
without fallback, fallback in every substep) and a random BF16 network.
"""
import numpy as np
import pytest

import oracle
from paper_2503_18616_gb300 import inputs
from sim_helpers import POS_TOL, gpu_positions, grid, make_sim, oracle_envs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ZERO_NORM = (np.zeros(15), np.ones(15), np.zeros(3), np.ones(3))


def _perturbed(sim, m, n_env, oenvs, seed):
    rest, w, _ = m
    V = len(rest)
    x = np.concatenate([inputs.perturbed_positions(rest, 3e-4, seed + e, inv_mass=w) for e in range(n_env)])
    v = np.random.default_rng(seed).normal(0, 0.01, x.shape)
    v[np.tile(w, n_env) == 0] = 0
    x32, v32 = x.astype(np.float32), v.astype(np.float32)
    sim.set_state(torch.from_numpy(x32).cuda(), torch.from_numpy(v32).cuda())
    for e, oe in oenvs.items():
        oe.set_state(x=x32[e * V:(e + 1) * V].astype(np.float64), v=v32[e * V:(e + 1) * V].astype(np.float64))


def test_recorded_features_and_targets_match_oracle():
    m = grid((9, 9, 5))
    p = inputs.default_params(radius=4e-3)
    n_env = 3
    sim = make_sim([m], p, n_env, seed=2)
    oenvs, om = oracle_envs([m], p, n_env, seed=2)
    _perturbed(sim, m, n_env, oenvs, 5)
    zeros = torch.zeros((n_env, 3), dtype=torch.float32, device="cuda")
    feats, targs = sim.record_step(10, actions=zeros)
    n_rows, off = sim.rows()
    feats, targs = feats.cpu().numpy(), targs.cpu().numpy()
    ext = om[0].extent
    V = om[0].V
    h = p["dt"] / p["substeps"]
    pos_cols = [0, 1, 2, 6, 7, 8, 12, 13, 14]
    vel_cols = [3, 4, 5, 9, 10, 11]
    for e, oe in oenvs.items():
        Fo, To = oe.step_record(10, action=np.zeros(3))
        Fg = feats[:, off[e]:off[e] + V, :]
        assert np.max(np.abs(Fg[..., pos_cols] - Fo[..., pos_cols])) <= POS_TOL * ext
        assert np.max(np.abs(Fg[..., vel_cols] - Fo[..., vel_cols])) <= POS_TOL * ext / h
        assert np.all(Fg[..., 15] == 0)
        assert np.max(np.abs(targs[:, off[e]:off[e] + V, :3] - To)) <= POS_TOL * ext
    x, _, _ = gpu_positions(sim)
    for e, oe in oenvs.items():
        assert np.max(np.abs(x[e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext


def _install(sim, params, norm):
    sim.set_network(params, *norm)


def _case_network(case):
    if case == "zero_no_fallback":
        params = {k: np.zeros_like(v) for k, v in oracle.mlp_init(0).items()}
        return params, ZERO_NORM, np.inf
    if case == "always_fallback":
        params = oracle.mlp_init(1)
        return params, (np.zeros(15), np.full(15, 1e-3), np.zeros(3), np.full(3, 1e-5)), -1.0
    params = oracle.mlp_init(2)
    rng = np.random.default_rng(3)
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.1, params[k].shape)
    return params, (np.zeros(15), np.full(15, 2e-3), np.zeros(3), np.full(3, 2e-7)), np.inf


@pytest.mark.parametrize("path", ["fused", "pipeline"])
@pytest.mark.parametrize("case", ["zero_no_fallback", "always_fallback", "random_network"])
def test_surrogate_step_matches_oracle(case, path):
    """Both implementations of the surrogate step: the fused kernel (state
    resident, network on the tensor cores of the same CTA) and the per-substep
    pipeline (features, network, substep launches)."""
    from paper_2503_18616_gb300 import ffsrl
    m = grid((9, 9, 5))
    p = inputs.default_params(radius=4e-3)
    n_env, steps = 3, 6
    flags = ffsrl.SCHED_SURROGATE_PIPELINE if path == "pipeline" else 0
    sim = make_sim([m], p, n_env, seed=4, schedule_flags=flags)
    oenvs, om = oracle_envs([m], p, n_env, seed=4)
    params, norm, thr = _case_network(case)
    _install(sim, params, norm)
    net = oracle.Net.from_params(params, *norm, bf16=True)
    fb = torch.zeros(n_env, dtype=torch.int32, device="cuda")
    for _ in range(steps):
        obs, rew, _ = sim.step_surrogate(thr if np.isfinite(thr) else 1e30, 10, fallbacks=fb)
    ofb, orew = {}, {}
    for e, oe in oenvs.items():
        ofb[e] = 0
        for _ in range(steps):
            o_obs, orew[e], _, f = oe.step_surrogate(net, thr, 10)
            ofb[e] += f
    sim.sync()
    x, v, tool = gpu_positions(sim)
    ext = om[0].extent
    V = om[0].V
    for e, oe in oenvs.items():
        ox, ov, oc = oe.state()
        assert np.max(np.abs(x[e * V:(e + 1) * V] - ox)) <= POS_TOL * ext, e
        assert np.array_equal(tool[e], oc)
        assert int(fb[e]) == ofb[e]
        assert abs(float(rew[e]) - orew[e]) <= POS_TOL * ext
    if case == "always_fallback":
        assert all(f == steps * p["substeps"] for f in ofb.values())
    else:
        assert all(f == 0 for f in ofb.values())


def test_fused_step_on_the_4096_env_mesh_matches_oracle():
    """The 17 x 17 x 9 block: 21 network tiles per substep with a ragged last
    tile (2601 = 20 x 128 + 41 rows); random network, no fallback, then a
    fallback in every substep."""
    m = grid((17, 17, 9))
    p = inputs.default_params()
    n_env, steps = 2, 3
    for case in ("random_network", "always_fallback"):
        sim = make_sim([m], p, n_env, seed=6)
        oenvs, om = oracle_envs([m], p, n_env, seed=6)
        params, norm, thr = _case_network(case)
        _install(sim, params, norm)
        net = oracle.Net.from_params(params, *norm, bf16=True)
        fb = torch.zeros(n_env, dtype=torch.int32, device="cuda")
        for _ in range(steps):
            sim.step_surrogate(thr if np.isfinite(thr) else 1e30, 10, fallbacks=fb)
        sim.sync()
        x, _, tool = gpu_positions(sim)
        V, ext = om[0].V, om[0].extent
        for e, oe in oenvs.items():
            f = 0
            for _ in range(steps):
                f += oe.step_surrogate(net, thr, 10)[3]
            assert np.max(np.abs(x[e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext, (case, e)
            assert np.array_equal(tool[e], oe.state()[2])
            assert int(fb[e]) == f


def test_mixed_rollout_steps_plain_and_warm_start_envs_together():
    """ffsrl_set_surrogate_envs: odd envs take the warm-start step inside
    ffsrl_step, even envs the plain step; every env matches the oracle's
    corresponding step, and switching the mask off restores plain stepping."""
    m = grid((9, 9, 5))
    p = inputs.default_params(radius=4e-3)
    n_env, steps = 4, 5
    sim = make_sim([m], p, n_env, seed=8)
    oenvs, om = oracle_envs([m], p, n_env, seed=8)
    params, norm, thr = _case_network("random_network")
    _install(sim, params, norm)
    net = oracle.Net.from_params(params, *norm, bf16=True)
    mask = np.array([e % 2 for e in range(n_env)], np.uint8)
    fb = torch.zeros(n_env, dtype=torch.int32, device="cuda")
    sim.set_surrogate_envs(mask, threshold=1e30, n_full=10, fallbacks=fb)
    for _ in range(steps):
        obs, rew, done = sim.step()
    sim.set_surrogate_envs(None)
    obs, rew, done = sim.step()            # one plain step for every env
    sim.sync()
    x, _, tool = gpu_positions(sim)
    V, ext = om[0].V, om[0].extent
    for e, oe in oenvs.items():
        for _ in range(steps):
            if mask[e]:
                oe.step_surrogate(net, thr, 10)
            else:
                oe.step()
        o_obs, o_rew, _ = oe.step()
        assert np.max(np.abs(x[e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext, e
        assert np.array_equal(tool[e], oe.state()[2])
        assert abs(float(rew[e]) - o_rew) <= POS_TOL * ext
        assert np.max(np.abs(obs[e].cpu().numpy() - o_obs)) <= POS_TOL * ext
    assert int(fb.sum()) == 0


def test_fallback_decided_per_env_and_substep():
    """A residual threshold between the per-substep residuals of the envs:
    some substeps fall back to the full solve and others keep the warm start.
    The threshold is chosen on the oracle so that no residual it checks lies
    within 1% of it (the float32 and float64 decisions then agree); the GPU
    must take the same decisions (equal fallback counts per env) and end
    within the position tolerance."""
    m = grid((9, 9, 5))
    p = inputs.default_params(radius=4e-3)
    n_env, steps, S = 4, 6, p["substeps"]
    params, norm, _ = _case_network("random_network")
    net = oracle.Net.from_params(params, *norm, bf16=True)

    def oracle_run(thr):
        oenvs, om = oracle_envs([m], p, n_env, seed=12)
        res, fbs = [], {}
        for e, oe in oenvs.items():
            fbs[e] = 0
            for _ in range(steps):
                r = np.zeros(S)
                fbs[e] += oe.step_surrogate(net, thr, 10, residuals=r)[3]
                res.append(r)
        return oenvs, om, np.concatenate(res), fbs

    _, _, r_free, _ = oracle_run(np.inf)
    thr = float(np.median(r_free))
    for _ in range(60):
        oenvs, om, r, fbs = oracle_run(thr)
        if np.min(np.abs(r / thr - 1.0)) > 0.01:
            break
        thr *= 1.013
    else:
        pytest.fail("no threshold with a 1% margin to every checked residual")
    total = sum(fbs.values())
    assert 0 < total < n_env * steps * S, fbs
    sim = make_sim([m], p, n_env, seed=12)
    _install(sim, params, norm)
    fb = torch.zeros(n_env, dtype=torch.int32, device="cuda")
    for _ in range(steps):
        sim.step_surrogate(thr, 10, fallbacks=fb)
    sim.sync()
    x, _, tool = gpu_positions(sim)
    V, ext = om[0].V, om[0].extent
    for e, oe in oenvs.items():
        assert int(fb[e]) == fbs[e], (e, int(fb[e]), fbs[e])
        assert np.max(np.abs(x[e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext, e
        assert np.array_equal(tool[e], oe.state()[2])


@pytest.mark.parametrize("shape", [(9, 9, 5), (17, 17, 9)])
def test_just_in_time_and_staged_kernels_give_the_same_bits(shape):
    """The fused warm-start step has two kernels: one builds each tile's input
    just in time and keeps the network outputs in TMEM until no later tile's
    features read their rows, the other stages inputs and corrections in
    global memory. Same operations, same rounding: equal bits, with and
    without fallbacks (threshold between the substeps' residuals)."""
    from paper_2503_18616_gb300 import ffsrl
    m = grid(shape)
    p = inputs.default_params(radius=4e-3)
    n_env, steps = 3, 4
    params, norm, _ = _case_network("random_network")
    out = {}
    for name, flags in (("jit", 0), ("staged", ffsrl.SCHED_WARM_STAGED)):
        sim = make_sim([m], p, n_env, seed=14, schedule_flags=flags)
        _install(sim, params, norm)
        fb = torch.zeros(n_env, dtype=torch.int32, device="cuda")
        res = torch.zeros(n_env, dtype=torch.float32, device="cuda")
        for k in range(steps):
            # the first steps without fallback, then a threshold that some substeps exceed
            thr = float("inf") if k < 2 else 8e-3
            obs, rew, _ = sim.step_surrogate(thr, 10, fallbacks=fb, residual=res)
        sim.sync()
        x, v, tool = sim.get_state()
        out[name] = (x.cpu().numpy(), v.cpu().numpy(), obs.cpu().numpy(), rew.cpu().numpy(), fb.cpu().numpy(),
                     res.cpu().numpy())
        sim.close()
    for a, b in zip(out["jit"], out["staged"]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(9, 9, 5), (17, 17, 9)])
def test_step_residual_matches_oracle(shape):
    """The residual the fallback decision reads (largest relative violation
    after the one iteration, W5), asked for at an infinite threshold so that
    nothing falls back: per env and step, the GPU's maximum over the step's
    substeps equals the oracle's within 1% (both read states that agree to
    the position tolerance; a relative violation moves by about the position
    error over the rest length)."""
    m = grid(shape)
    p = inputs.default_params(radius=4e-3)
    n_env, steps, S = 3, 8, p["substeps"]
    params, norm, _ = _case_network("random_network")
    net = oracle.Net.from_params(params, *norm, bf16=True)
    oenvs, _ = oracle_envs([m], p, n_env, seed=21)
    sim = make_sim([m], p, n_env, seed=21)
    _install(sim, params, norm)
    res = torch.zeros(n_env, dtype=torch.float32, device="cuda")
    for k in range(steps):
        res.zero_()
        sim.step_surrogate(float("inf"), 10, residual=res)
        g = res.cpu().numpy()
        for e, oe in oenvs.items():
            r = np.zeros(S)
            oe.step_surrogate(net, float("inf"), 10, residuals=r)
            assert r.max() > 0
            assert abs(g[e] - r.max()) <= 1e-2 * r.max(), (k, e, float(g[e]), float(r.max()))


@pytest.mark.parametrize("pinned", ["top_layer", "all"])
def test_warm_start_with_other_pinned_sets(pinned):
    """The fused kernel skips leading 128-slot tiles that hold pinned vertices
    only (their corrections are never applied). With the top layer pinned
    instead of the bottom one no tile is skipped at the start; with every
    vertex pinned every tile is, and nothing may move. The just-in-time and
    staged kernels (the latter runs every tile) must give the same bits, and
    the oracle's surrogate step the same positions within the tolerance."""
    from paper_2503_18616_gb300 import ffsrl
    rest, w, tets = grid((17, 17, 9))
    w = w.copy()
    if pinned == "top_layer":
        w[:] = 1.0 / inputs.MASS
        w[rest[:, 2] == rest[:, 2].max()] = 0.0
    else:
        w[:] = 0.0
    m = (rest, w, tets)
    p = inputs.default_params(radius=4e-3)
    n_env, steps = 2, 3
    params, norm, _ = _case_network("random_network")
    out = {}
    for name, flags in (("jit", 0), ("staged", ffsrl.SCHED_WARM_STAGED)):
        sim = make_sim([m], p, n_env, seed=16, schedule_flags=flags)
        _install(sim, params, norm)
        x0, _, _ = sim.get_state()
        x0 = x0.cpu().numpy()
        for _ in range(steps):
            sim.step_surrogate(float("inf"), 10)
        sim.sync()
        x, v, _ = sim.get_state()
        out[name] = (x.cpu().numpy(), v.cpu().numpy())
        sim.close()
    assert np.array_equal(out["jit"][0], out["staged"][0]) and np.array_equal(out["jit"][1], out["staged"][1])
    if pinned == "all":
        assert np.array_equal(out["jit"][0], x0) and not out["jit"][1].any()
        return
    net = oracle.Net.from_params(params, *norm, bf16=True)
    oenvs, om = oracle_envs([m], p, n_env, seed=16)
    V, ext = om[0].V, om[0].extent
    for e, oe in oenvs.items():
        for _ in range(steps):
            oe.step_surrogate(net, float("inf"), 10)
        assert np.max(np.abs(out["jit"][0][e * V:(e + 1) * V] - oe.state()[0])) <= POS_TOL * ext
