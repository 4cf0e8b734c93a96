"""Writes oracle_regression.json: sampled outputs of the FP64 oracle on small
fixed cases, so that a later change to the oracle's arithmetic shows up as a
failing regression test (tests/test_oracle_regression.py). Calls only the
oracle and the seeded input generators. Run from the repository root:

    python tests/golden/make_oracle_regression.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2503_18616_gb300 import inputs  # noqa: E402

CASES = {
    # the plain step: sphere tool, 10 substeps x 1 iteration, device-style draws
    "block9x9x5_sphere_20steps": {"shape": (9, 9, 5), "params": {}, "steps": 20, "seed": 3, "env": 1},
    # two iterations (multipliers carried), stiffer distance compliance
    "block9x9x5_iter2_20steps": {"shape": (9, 9, 5), "params": {"iterations": 2, "alpha_d": 1e-7}, "steps": 20,
                                 "seed": 4, "env": 0},
    # the paper's Jacobi solver
    "block5x5x3_jacobi_10steps": {"shape": (5, 5, 3), "params": {"solver": 1, "iterations": 4, "n_obs": 8},
                                  "steps": 10, "seed": 5, "env": 2},
    # the grasper pressed down into the tissue
    "block9x9x5_grasper_12steps": {"shape": (9, 9, 5), "params": {"tool_model": 1}, "steps": 12, "seed": 6,
                                   "env": 0, "down": True},
    # tissue connected to its base
    "stacked9x9x3x3_conn_12steps": {"stacked": (9, 9, 3, 3), "params": {"conn_radius": 6e-3}, "steps": 12,
                                    "seed": 7, "env": 0},
}


def run(case):
    if "stacked" in case:
        mesh = inputs.stacked_blocks(*case["stacked"], gap=1e-3)
    else:
        mesh = inputs.grid_block(*case["shape"])
    p = inputs.default_params(**case["params"])
    om = oracle.Mesh(*mesh, conn_radius=p.get("conn_radius", 0.0))
    e = oracle.Env(om, p)
    e.reset(case["seed"], case["env"])
    rewards = []
    for k in range(case["steps"]):
        a = np.array([0.0, 0.0, -1.0]) if case.get("down") and k < case["steps"] // 2 else None
        _, r, _ = e.step(a)
        rewards.append(float(r))
    x, v, c = e.state()
    idx = np.linspace(0, len(x) - 1, 12).round().astype(int)
    return {"rewards": rewards, "tool": c.tolist(), "sample_ids": idx.tolist(),
            "x_sample": x[idx].tolist(), "v_sample": v[idx].tolist(),
            "x_sum": float(np.sum(x)), "x_abs_sum": float(np.sum(np.abs(x - mesh[0]))),
            "contacts": [int(i) for i in e.ints()["contacts"]]}


def main():
    out = {name: run(case) for name, case in CASES.items()}
    path = os.path.join(ROOT, "tests", "golden", "oracle_regression.json")
    with open(path, "w") as f:
        json.dump({"note": "written by tests/golden/make_oracle_regression.py from the FP64 oracle",
                   "cases": out}, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
