"""Training driver of the learned warm-start network.

The warm-start is not in the FF-SRL paper: it is a per-vertex network
(15 -> 64 -> ReLU -> 64 -> ReLU -> 3, BF16 on the tensor cores) that predicts
the position correction of the full constraint solve from features of the
predicted state, so that one iteration can replace several. Training data come
from the simulator itself: ffsrl_record_step runs the plain full solve and
writes, for every vertex row and substep, the features and the target
correction. Every arithmetic step (recording, normalisation, forward,
backward, Adam) runs in the library's CUDA kernels; this module only
schedules them.
"""
from __future__ import annotations

import math
import time

import numpy as np

N_IN, N_HID, N_OUT = 15, 64, 3


def init_network(seed: int) -> dict:
    """He-uniform weights and zero biases (output-major layout)."""
    rng = np.random.default_rng(seed)

    def layer(n_out, n_in):
        lim = math.sqrt(6.0 / n_in)
        return rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)

    W1, b1 = layer(N_HID, N_IN)
    W2, b2 = layer(N_HID, N_HID)
    W3, b3 = layer(N_OUT, N_HID)
    W3 *= 0.1   # start close to "no correction"
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def row_weights(sim, meshes, env_mesh=None):
    """Float32 tensor [rows]: 1 for the free vertices of every env, 0 for
    pinned vertices and padding rows."""
    import torch
    n_rows, off = sim.rows()
    w = np.zeros(n_rows, np.float32)
    for e in range(sim.n_env):
        rest, inv_mass, _ = meshes[0 if env_mesh is None else int(env_mesh[e])]
        w[off[e]:off[e] + len(rest)] = (np.asarray(inv_mass) > 0).astype(np.float32)
    return torch.from_numpy(w).to(sim.device)




def train(sim, meshes, n_full: int = 10, env_substeps: int = 200_000, lr: float = 1e-3, epochs: int = 2,
          seed: int = 0, env_mesh=None, log=None, lr_final: float | None = None):
    """Trains the network of `sim` on trajectories of its own full solve.

    Each ffsrl_record_step advances every env one step with the n_full
    iteration solve and records all vertex rows of all substeps; each substep's
    rows form one batch, visited `epochs` times with Adam. Recording stops once
    env_substeps env-substeps have been generated. With lr_final the learning
    rate follows a cosine from lr down to lr_final over the Adam steps, else it
    stays lr. Returns a summary dict with the parameters, normalisation and
    loss history (normalised MSE)."""
    import torch
    t0 = time.perf_counter()
    w = row_weights(sim, meshes, env_mesh)
    wsum = float(w.sum().item())
    S = sim.params["substeps"]
    sim.reset(seed)
    F, T = sim.record_step(n_full)
    # the frozen normalisation of the first recorded step's rows (device kernel)
    norm = sim.network_normalisation(F, T, w.expand(S, -1).contiguous())
    sim.set_network(init_network(seed), *norm)
    loss = torch.zeros(1, dtype=torch.float32, device=sim.device)
    losses = []
    n_records = max(1, math.ceil(env_substeps / (sim.n_env * S)))
    n_adam = n_records * epochs * S
    done_substeps = sim.n_env * S
    k_adam = 0

    def rate():
        if lr_final is None:
            return lr
        return lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k_adam / max(1, n_adam - 1)))
    for rec in range(n_records):
        if rec > 0:
            if rec % 50 == 0:
                sim.reset(seed + rec)      # fresh episodes: new targets, observed vertices, actions
            sim.record_step(n_full, features=F, targets=T)
            done_substeps += sim.n_env * S
        for _ in range(epochs):
            for s in range(S):
                sim.train_network(F[s], T[s], w, wsum, rate(), loss)
                k_adam += 1
        losses.append(float(loss.item()) / (3 * wsum))
        if log:
            log(f"record {rec + 1}/{n_records}: loss {losses[-1]:.4e}")
    sim.sync()
    return {"params": sim.get_network(), "norm": norm, "losses": losses, "env_substeps": done_substeps,
            "adam_steps": n_adam, "seconds": time.perf_counter() - t0}
