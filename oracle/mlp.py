"""FP64 oracle of the per-vertex warm-start network (test infrastructure only).

The learned warm-start is not in the FF-SRL paper (arXiv 2503.18616); it is a
network added on top of the paper's XPBD substep: a per-vertex
multilayer perceptron 15 -> 64 -> ReLU -> 64 -> ReLU -> 3 that predicts the
position correction of the constraint solve. This module is the plain numpy
definition used to check the GPU kernels: forward, the backward pass of the
mean-squared-error loss, and Adam (Kingma & Ba, ICLR 2015, Algorithm 1).

Layout: weights are stored output-major, ``W1[64, 15]``, ``W2[64, 64]``,
``W3[3, 64]``; biases ``b1[64]``, ``b2[64]``, ``b3[3]``. A batch is ``F[n, 15]``.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 15, 64, 3

__all__ = ["N_IN", "N_HID", "N_OUT", "mlp_init", "mlp_forward", "mlp_loss", "mlp_backward",
           "adam_step", "bf16_round", "normalisation"]


def mlp_init(seed: int, scale: float = 1.0) -> dict:
    """He-uniform initial weights (any seeded draw is a valid start)."""
    rng = np.random.default_rng(seed)

    def lin(n_out, n_in):
        lim = scale * np.sqrt(6.0 / n_in)
        return rng.uniform(-lim, lim, size=(n_out, n_in)), np.zeros(n_out)

    W1, b1 = lin(N_HID, N_IN)
    W2, b2 = lin(N_HID, N_HID)
    W3, b3 = lin(N_OUT, N_HID)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


def mlp_forward(p: dict, F: np.ndarray):
    """Returns the output y[n, 3] and the activations the backward pass needs."""
    F = np.asarray(F, dtype=np.float64)
    z1 = F @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, {"F": F, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def mlp_loss(y: np.ndarray, target: np.ndarray) -> float:
    """Mean over samples and components of the squared error."""
    return float(np.mean((y - target) ** 2))


def mlp_backward(p: dict, cache: dict, y: np.ndarray, target: np.ndarray) -> dict:
    """Gradients of ``mlp_loss`` with respect to every parameter."""
    n = y.shape[0]
    dy = 2.0 * (y - target) / (n * N_OUT)
    g = {"W3": dy.T @ cache["h2"], "b3": dy.sum(axis=0)}
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["F"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; t is the 1-based step count."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mhat = m[k] / (1 - beta1 ** t)
        vhat = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)


def normalisation(F: np.ndarray, T: np.ndarray, w: np.ndarray):
    """Frozen normalisation of the network's inputs and outputs: per column,
    the mean and the population standard deviation (divisor n) over the rows
    whose weight is positive; a column with zero spread gets std 1. F holds
    at least 15 feature columns, T at least 3 target columns.

    Returns (in_mean[15], in_std[15], out_mean[3], out_std[3])."""
    sel = np.asarray(w).reshape(-1) > 0
    f = np.asarray(F, dtype=np.float64)[sel][:, :N_IN]
    t = np.asarray(T, dtype=np.float64)[sel][:, :N_OUT]
    out = []
    for a in (f, t):
        mean = a.sum(axis=0) / len(a)
        std = np.sqrt(((a - mean) ** 2).sum(axis=0) / len(a))
        out += [mean, np.where(std > 0, std, 1.0)]
    return out[0], out[1], out[2], out[3]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)
