"""Shared helpers of the parity tests: build the CUDA simulator and the oracle
from the same seeded inputs and compare their outputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2503_18616_gb300 import inputs

POS_TOL = 1e-5          # max |x_gpu - x_oracle| / extent (FP32 path vs FP64 oracle)


def make_sim(meshes, params, n_env, env_mesh=None, env_compliance=None, block_threads=0, seed=0,
             schedule_flags=0):
    from paper_2503_18616_gb300 import build, ffsrl
    build.build()
    sim = ffsrl.Sim(meshes, params, n_env, env_mesh=env_mesh, env_compliance=env_compliance,
                    block_threads=block_threads, schedule_flags=schedule_flags)
    sim.reset(seed)
    return sim


def oracle_envs(meshes, params, n_env, env_mesh=None, env_compliance=None, seed=0, envs=None):
    """Oracle environments for the listed env ids (default: all)."""
    envs = range(n_env) if envs is None else envs
    om = [oracle.Mesh(*m) for m in meshes]
    out = {}
    for e in envs:
        mi = 0 if env_mesh is None else int(env_mesh[e])
        p = dict(params)
        if env_compliance is not None:
            p["alpha_d"] = float(env_compliance[e])
        oe = oracle.Env(om[mi], p)
        oe.reset(seed, e)
        out[e] = oe
    return out, om


def packed_offsets(meshes, n_env, env_mesh=None):
    sizes = [len(meshes[0 if env_mesh is None else int(env_mesh[e])][0]) for e in range(n_env)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def gpu_positions(sim):
    x, v, tool = sim.get_state()
    return x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64), tool.cpu().numpy()


def max_rel_err(a, b, extent):
    return float(np.max(np.abs(a - b)) / extent) if a.size else 0.0


def grid(shape):
    return inputs.grid_block(*shape)
