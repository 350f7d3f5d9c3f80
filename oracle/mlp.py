"""FP64 oracle of the cost-model network -- TEST INFRASTRUCTURE.

Only tests and the smoke check use this module.  The paper picks the rows to
rewrite by hand (Sec. IV); the library replaces that choice by a small
network that predicts the solve time of a rewrite choice.  This module is the
plain textbook definition of that network, used to check the library's own
forward, backward and optimizer kernels:

    z1 = X W1 + b1,  h1 = relu(z1)          W1: [F, H]
    z2 = h1 W2 + b2, h2 = relu(z2)          W2: [H, H]
    y  = h2 W3 + b3                          W3: [H, 1]
    loss = mean((y - target)^2)

relu'(0) is taken as 0.  Adam (Kingma & Ba, 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(n_in: int, hidden: int = 64, seed: int = 0) -> dict:
    """He-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)

    def he(fan_in, shape):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, shape)

    return dict(W1=he(n_in, (n_in, hidden)), b1=np.zeros(hidden),
                W2=he(hidden, (hidden, hidden)), b2=np.zeros(hidden),
                W3=he(hidden, (hidden, 1)), b3=np.zeros(1))


def forward(p: dict, X: np.ndarray) -> tuple[np.ndarray, dict]:
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ p["W3"] + p["b3"])[:, 0]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)


def loss(p: dict, X: np.ndarray, target: np.ndarray) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - target) ** 2))


def loss_and_grads(p: dict, X: np.ndarray, target: np.ndarray):
    y, c = forward(p, X)
    n = y.shape[0]
    dy = (2.0 / n) * (y - target)[:, None]          # [N, 1]
    g = {}
    g["W3"] = c["h2"].T @ dy
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"].T) * (c["z2"] > 0.0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (c["z1"] > 0.0)
    g["W1"] = c["X"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - target) ** 2)), g


def adam_init(p: dict) -> dict:
    return dict(t=0, m={k: np.zeros_like(v) for k, v in p.items()},
                v={k: np.zeros_like(v) for k, v in p.items()})


def adam_step(p: dict, g: dict, st: dict, lr: float = 1e-3,
              beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    st["t"] += 1
    t = st["t"]
    for k in PARAM_NAMES:
        st["m"][k] = beta1 * st["m"][k] + (1.0 - beta1) * g[k]
        st["v"][k] = beta2 * st["v"][k] + (1.0 - beta2) * g[k] * g[k]
        mh = st["m"][k] / (1.0 - beta1 ** t)
        vh = st["v"][k] / (1.0 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
