"""Pins of the oracle's two options beyond the default step.

Jacobi iterations (the paper's own parallel scheme, Sec. III-A): every
constraint steps from the iteration's start positions and each vertex moves
by the sum of its corrections divided by the number of constraints that
contain it. Pinned by properties that a plausible mistake breaks: the rest
state is a fixed point, the result does not depend on the constraint order
(Gauss-Seidel does), a vertex moves to the average of what each constraint
alone would do (each single projection being pinned elsewhere), repeated
iterations drive every constraint to zero, rotation equivariance.

Auto-reset (the episode handling of Sec. III-B): an env whose step reported
done starts its next episode at its next step, equal to a fresh reset with
the episode's seed followed by one step.
"""
import numpy as np

import oracle
from paper_2503_18616_gb300 import inputs


def params(**over):
    return inputs.default_params(**over)


def _shuffled(tets, seed):
    return tets[np.random.default_rng(seed).permutation(len(tets))]


def test_jacobi_rest_state_is_a_fixed_point():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    e = oracle.Env(oracle.Mesh(rest, w, tets), params(solver=1, gravity=(0.0, 0.0, 0.0), radius=0.0, iterations=3))
    e.reset(1)
    e.run(4, want_obs=False)
    x, v, _ = e.state()
    assert np.array_equal(x, rest) and np.all(v == 0)


def test_jacobi_does_not_depend_on_constraint_order_but_gauss_seidel_does():
    rest, w, tets = inputs.grid_block(5, 4, 3)
    x0 = inputs.perturbed_positions(rest, 4e-4, 3, inv_mass=w)
    out = {}
    for solver in (0, 1):
        for order in (0, 1):
            t = tets if order == 0 else _shuffled(tets, 11)
            e = oracle.Env(oracle.Mesh(rest, w, t), params(solver=solver, radius=0.0, n_obs=4, iterations=2))
            e.reset(0)
            e.set_state(x=x0, v=np.zeros_like(x0))
            e.run(3, want_obs=False)
            out[solver, order] = e.state()[0]
    assert np.max(np.abs(out[1, 0] - out[1, 1])) < 1e-15 * 1e3    # sums in another order only
    assert np.max(np.abs(out[0, 0] - out[0, 1])) > 1e-9            # another colouring, another result


def test_jacobi_moves_a_vertex_to_the_average_of_the_single_projections():
    """One tet with three pinned vertices: the free vertex belongs to three
    edges and the tet (n = 4); one Jacobi iteration moves it by the mean of
    the four moves each constraint alone makes from the same start."""
    s = inputs.CELL
    rest = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], dtype=np.float64)
    w = np.array([0.0, 0.0, 0.0, 1.0 / inputs.MASS])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    m = oracle.Mesh(rest, w, tets)
    p = params(solver=1, gravity=(0.0, 0.0, 0.0), radius=0.0, n_obs=1, substeps=1, iterations=1,
               alpha_d=0.0, alpha_v=0.0)
    e = oracle.Env(m, p)
    e.reset(0)
    x0 = rest.copy()
    x0[3] += np.array([4e-4, -7e-4, 9e-4])
    e.set_state(x=x0, v=np.zeros_like(x0))
    e.step()
    xd = e.state()[0][3]
    moves = []
    for a in (0, 1, 2):   # edges (a, 3), rest length |rest_a - rest_3|
        d = np.linalg.norm(rest[a] - rest[3])
        _, xb, _, _ = oracle.project_edge(x0[a], x0[3], w[a], w[3], d, 0.0)
        moves.append(xb - x0[3])
    V0 = abs(np.dot(np.cross(rest[1] - rest[0], rest[2] - rest[0]), rest[3] - rest[0])) / 6
    xs, _, _ = oracle.project_tet([x0[0], x0[1], x0[2], x0[3]], w, V0, 0.0)
    moves.append(xs[3] - x0[3])
    expect = x0[3] + np.mean(moves, axis=0)
    assert np.allclose(xd, expect, rtol=0, atol=1e-15)
    assert np.array_equal(e.state()[0][:3], rest[:3])


def test_jacobi_iterations_drive_the_constraints_to_zero():
    rest, _, tets = inputs.grid_block(4, 3, 3, pin_bottom=False)
    w = np.full(len(rest), 1.0 / inputs.MASS)
    m = oracle.Mesh(rest, w, tets)
    p = params(solver=1, gravity=(0.0, 0.0, 0.0), radius=0.0, n_obs=4, substeps=1, iterations=1600,
               alpha_d=0.0, alpha_v=0.0)
    e = oracle.Env(m, p)
    e.reset(0)
    x0 = inputs.perturbed_positions(rest, 3e-4, 7)
    e.set_state(x=x0, v=np.zeros_like(x0))
    before = e.residual()
    e.step()
    after = e.residual()
    assert before > 1e-2 and after < 1e-8, (before, after)


def test_jacobi_is_rotation_equivariant():
    rest, _, tets = inputs.grid_block(4, 3, 3, pin_bottom=False)
    w = np.full(len(rest), 1.0 / inputs.MASS)
    m = oracle.Mesh(rest, w, tets)
    p = params(solver=1, gravity=(0.0, 0.0, 0.0), radius=0.0, n_obs=4, iterations=2)
    rng = np.random.default_rng(4)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    x0 = inputs.perturbed_positions(rest, 1e-3, 9)
    v0 = rng.normal(0, 0.05, rest.shape)
    outs = []
    for R in (np.eye(3), q):
        e = oracle.Env(m, p)
        e.reset(0)
        e.set_state(x=x0 @ R.T, v=v0 @ R.T)
        e.run(4, want_obs=False)
        outs.append(e.state()[0])
    assert np.allclose(outs[0] @ q.T, outs[1], atol=1e-12)


def test_auto_reset_starts_the_next_episode_like_a_fresh_reset():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    m = oracle.Mesh(rest, w, tets)
    p = params(max_steps=3, auto_reset=1)
    seed, env = 5, 2
    e = oracle.Env(m, p)
    e.reset(seed, env)
    dones = [e.step()[2] for _ in range(3)]
    assert dones == [0, 0, 1]
    obs, rew, done = e.step()                 # first step of episode 1
    fresh = oracle.Env(m, p)
    fresh.reset(oracle.episode_seed(seed, 1), env)
    f_obs, f_rew, f_done = fresh.step()
    assert np.array_equal(obs, f_obs) and rew == f_rew and done == f_done
    for a, b in zip(e.state(), fresh.state()):
        assert np.array_equal(a, b)
    ints, f_ints = e.ints(), fresh.ints()
    assert ints["t"] == 1 and ints["episode"] == 1
    assert ints["target"] == f_ints["target"] and np.array_equal(ints["obs_ids"], f_ints["obs_ids"])
    assert oracle.episode_seed(seed, 1) == oracle.sm64(seed, (1 << 40) + 1)


def test_without_auto_reset_done_envs_keep_stepping():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    e = oracle.Env(oracle.Mesh(rest, w, tets), params(max_steps=3))
    e.reset(5, 2)
    dones = [e.step()[2] for _ in range(5)]
    assert dones == [0, 0, 1, 1, 1] and e.ints()["t"] == 5 and e.ints()["episode"] == 0


def test_success_resets_every_step_when_always_successful():
    rest, w, tets = inputs.grid_block(9, 9, 5)
    e = oracle.Env(oracle.Mesh(rest, w, tets), params(success_dist=1.0, auto_reset=1))
    e.reset(3, 0)
    for k in range(4):
        assert e.step()[2] == 1
    assert e.ints()["episode"] == 3 and e.ints()["t"] == 1
