"""Seeded synthetic inputs shared by the simulator tests, the benchmark and the
oracle checks.

This module holds no arithmetic of the method: it only draws the tet meshes,
initial states, actions and per-environment compliances that both sides are
given. The mesh is a block of cubes, each split into five tets, shaped like the
tissue blocks of the paper's tissue-manipulation scene (Sec. IV); the paper's
own meshes are not published, so these stand in for them.

Conventions:
  * vertex id = (k * ny + j) * nx + i for grid point (i, j, k);
  * cell size ``spacing`` (5 mm by default), x and y centred on 0, bottom face
    at z = 0; the bottom face is pinned (inverse mass 0);
  * the five-tet split alternates with cell parity so that neighbouring cells
    share face diagonals (a conforming mesh): in a cell whose i+j+k is even the
    central tet takes the four corners with an odd offset sum, in an odd cell
    the four with an even offset sum; the other four corners each get a corner
    tet made of the corner and its three axis neighbours in the cell. Each cell
    emits its central tet first, then the corner tets.
"""
from __future__ import annotations

import math

import numpy as np

CELL = 5e-3          # grid spacing in metres
MASS = 1e-3          # particle mass in kg


def grid_block(nx: int, ny: int, nz: int, spacing: float = CELL, mass: float = MASS,
               pin_bottom: bool = True):
    """Vertex grid of nx x ny x nz points split into 5 (nx-1)(ny-1)(nz-1) tets.

    Returns (rest [V,3] float64, inv_mass [V] float64, tets [T,4] int32)."""
    if min(nx, ny, nz) < 2:
        raise ValueError("need at least 2 points per axis")
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # order by id = (k*ny + j)*nx + i
    idx = lambda i, j, k: (k * ny + j) * nx + i  # noqa: E731
    V = nx * ny * nz
    rest = np.zeros((V, 3), dtype=np.float64)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                rest[idx(i, j, k)] = ((i - (nx - 1) / 2) * spacing,
                                      (j - (ny - 1) / 2) * spacing,
                                      k * spacing)
    inv_mass = np.full(V, 1.0 / mass, dtype=np.float64)
    if pin_bottom:
        inv_mass[rest[:, 2] == 0.0] = 0.0
    corners = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    tets = []
    for k in range(nz - 1):
        for j in range(ny - 1):
            for i in range(nx - 1):
                central_parity = 1 if (i + j + k) % 2 == 0 else 0
                cid = lambda o: idx(i + o[0], j + o[1], k + o[2])  # noqa: E731
                central = [o for o in corners if sum(o) % 2 == central_parity]
                tips = [o for o in corners if sum(o) % 2 != central_parity]
                tets.append([cid(o) for o in central])
                for o in tips:
                    nb = [(1 - o[0], o[1], o[2]), (o[0], 1 - o[1], o[2]), (o[0], o[1], 1 - o[2])]
                    tets.append([cid(o)] + [cid(q) for q in nb])
    del ii, jj, kk
    return rest, inv_mass, np.asarray(tets, dtype=np.int32)


def stacked_blocks(nx: int, ny: int, nz_base: int, nz_top: int, gap: float = 0.0, spacing: float = CELL,
                   mass: float = MASS):
    """Two objects in one mesh: a base block (an organ, bottom face pinned) and
    a tissue block of the same footprint laid on it `gap` above its top face,
    free (its bottom face unpinned), for the tissue-connection scene of the
    paper's retraction task (Sec. III-A, Sec. IV). Base vertices come first.

    Returns (rest [V,3], inv_mass [V], tets [T,4])."""
    r0, w0, t0 = grid_block(nx, ny, nz_base, spacing, mass, pin_bottom=True)
    r1, w1, t1 = grid_block(nx, ny, nz_top, spacing, mass, pin_bottom=False)
    r1 = r1.copy()
    r1[:, 2] += r0[:, 2].max() + gap
    return (np.concatenate([r0, r1]), np.concatenate([w0, w1]),
            np.concatenate([t0, t1 + len(r0)]).astype(np.int32))


def two_tet_mesh(spacing: float = CELL, mass: float = MASS):
    """Two tets sharing one face (5 vertices, 9 edges), no pinned vertex."""
    s = spacing
    rest = np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s], [s, s, s]], dtype=np.float64)
    inv_mass = np.full(5, 1.0 / mass)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    return rest, inv_mass, tets


def block_shape_for(v_target: float):
    """Grid with aspect 2:2:1 whose vertex count is near v_target.

    Solves (2s+1)^2 (s+1) = v_target for s; cells nz = max(1, round(s)) and
    nx = ny = max(1, round(2s)); returns vertex counts (nx+1, ny+1, nz+1)."""
    lo, hi = 0.0, 1e4
    for _ in range(200):
        mid = (lo + hi) / 2
        if (2 * mid + 1) ** 2 * (mid + 1) < v_target:
            lo = mid
        else:
            hi = mid
    s = (lo + hi) / 2
    cz = max(1, int(round(s)))
    cxy = max(1, int(round(2 * s)))
    return cxy + 1, cxy + 1, cz + 1


def uneven_sizes(n_env: int, v_min: float, v_max: float, seed: int):
    """Per-env vertex targets drawn log-uniformly from [v_min, v_max]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(v_min), math.log(v_max), size=n_env))


def uneven_batch(n_env: int, v_min: float, v_max: float, seed: int):
    """Distinct grid shapes and the env -> shape map for an uneven batch.

    Returns (shapes: list of (nx, ny, nz), env_mesh: int32 [n_env])."""
    targets = uneven_sizes(n_env, v_min, v_max, seed)
    shapes: list = []
    env_mesh = np.zeros(n_env, dtype=np.int32)
    for e, v in enumerate(targets):
        sh = block_shape_for(v)
        if sh not in shapes:
            shapes.append(sh)
        env_mesh[e] = shapes.index(sh)
    return shapes, env_mesh


def compliance_draws(n_env: int, lo: float, hi: float, seed: int):
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(lo, hi, size=n_env)


def random_actions(n_steps: int, n_env: int, seed: int):
    """Uniform actions in [-1, 1]^3, float32-representable, [n_steps, n_env, 3]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_steps, n_env, 3)).astype(np.float32).astype(np.float64)


def perturbed_positions(rest: np.ndarray, amplitude: float, seed: int, inv_mass=None):
    """Rest positions plus uniform noise of the given amplitude (pinned rows kept)."""
    rng = np.random.default_rng(seed)
    x = rest + rng.uniform(-amplitude, amplitude, size=rest.shape)
    if inv_mass is not None:
        x[inv_mass == 0] = rest[inv_mass == 0]
    return x


def default_params(spacing: float = CELL, **over) -> dict:
    """Parameter set of the tissue workloads (dt 1/60 s, 10 substeps x 1
    iteration, compliance 1e-6 for distance and 0 for volume, sphere tool of
    radius half a cell moving 2 mm per unit action, 64 observed surface
    vertices, reward = -distance to the target vertex)."""
    p = {
        "dt": 1.0 / 60.0,
        "substeps": 10,
        "iterations": 1,
        "gravity": (0.0, 0.0, -9.81),
        "alpha_d": 1e-6,
        "alpha_v": 0.0,
        "radius": 0.5 * spacing,
        "action_scale": 2e-3,
        "margin_xy": 2.0 * spacing,
        "margin_below": 1.0 * spacing,
        "margin_above": 6.0 * spacing,
        "w_l": -1.0,
        "w_d": 0.0,
        "w_s": 0.0,
        "success_dist": 3e-3,
        "n_obs": 64,
        "max_steps": 0,
        "solver": 0,        # 0 colour Gauss-Seidel, 1 Jacobi with averaging (the paper's GPU scheme)
        "auto_reset": 0,    # 1: a done env starts a new episode at its next step
        # tool: 0 sphere proxy (the default), 1 the paper's three-capsule grasper through a remote
        # centre of motion 8 cells above the top face (shaft radius half a cell, clamps two cells
        # long, a quarter cell thick, opened 10 degrees)
        "tool_model": 0,
        "rcm_height": 8.0 * spacing,
        "shaft_radius": 0.5 * spacing,
        "clamp_length": 2.0 * spacing,
        "clamp_radius": 0.25 * spacing,
        "clamp_angle": math.radians(10.0),
        "grasp_radius": 0.5 * spacing,   # dragging: nearest free vertex within this of the clamp end
        "conn_radius": 0.0,  # > 0: tissue connections between the objects of a mesh, up to this rest distance
    }
    p.update(over)
    return p


# Workloads of the benchmark and the parity tests, by what they are.
WORKLOADS = {
    "block9x9x5_1env_100steps": {"shape": (9, 9, 5), "n_env": 1, "steps": 100},
    "block17x17x9_4096env_1000steps": {"shape": (17, 17, 9), "n_env": 4096, "steps": 1000},
    "uneven500-20000_1024env_500steps": {"n_env": 1024, "v_range": (500, 20000), "steps": 500,
                                          "alpha_range": (1e-7, 1e-5)},
    # the paper's Jacobi iterations against colour Gauss-Seidel at equal error
    "solvers_block17x17x9_4096env": {"shape": (17, 17, 9), "n_env": 4096, "steps": 100, "solvers": True},
    # full device-resident rollout: odd envs take the warm-start step (network
    # + 1 iteration, fallback to the 10-iteration solve), even envs the plain step
    "block17x17x9_16384env_2000steps": {"shape": (17, 17, 9), "n_env": 16384, "steps": 2000, "mixed": True,
                                        "train_envs": 512, "train_env_substeps": 200_000, "n_full": 10},
    # the paper's tissue-retraction scene: a 17x17x5 tissue block connected (6 mm) to a
    # 17x17x5 base block 1 mm below it, the three-capsule grasper with closed clamps
    # (1 degree) dragging the tissue along the device-drawn random walk
    "retraction_stacked17x17x5x5_4096env": {"stacked": (17, 17, 5, 5), "gap": 1e-3, "n_env": 4096, "steps": 1000,
                                            "params": {"tool_model": 1, "conn_radius": 6e-3,
                                                       "clamp_angle": math.radians(1.0)}},
    # learned warm-start: trained on 200k full-solve (10 iteration) env-substeps,
    # then network + 1 iteration with residual fallback, compared with plain k
    "warmstart_block17x17x9_4096env": {"shape": (17, 17, 9), "n_env": 4096, "steps": 200, "warmstart": True,
                                       "train_envs": 512, "train_env_substeps": 200_000, "n_full": 10,
                                       "threshold": 1e-4},
}
