"""FP64 reference of the path cost model: a 3-layer MLP on step features.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper motivates a cost model by noting that a path with more flops can
run faster (Sec. 4.3 discussion of Table 2) but gives no model; this is the
plain definition of the network the GPU trains:

    z1 = x W1 + b1,  a1 = relu(z1)
    z2 = a1 W2 + b2, a2 = relu(z2)
    y  = a2 W3 + b3                     (one output: predicted log step time)
    loss = mean over the batch of (y - t)^2

with W1: [d_in][h], W2: [h][h], W3: [h][1], gradients by the chain rule, and
Adam (Kingma & Ba, 2015) with bias correction:
    m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
    p <- p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(d_in: int, hidden: int, seed: int) -> dict:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)

    def u(fan_in, shape):
        b = np.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, size=shape)

    return {"W1": u(d_in, (d_in, hidden)), "b1": np.zeros(hidden),
            "W2": u(hidden, (hidden, hidden)), "b2": np.zeros(hidden),
            "W3": u(hidden, (hidden, 1)), "b3": np.zeros(1)}


def forward(P: dict, X: np.ndarray):
    z1 = X @ P["W1"] + P["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ P["W2"] + P["b2"]
    a2 = np.maximum(z2, 0.0)
    y = (a2 @ P["W3"] + P["b3"])[:, 0]
    return y, (X, z1, a1, z2, a2)


def loss(P: dict, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(P, X)
    return float(np.mean((y - t) ** 2))


def gradients(P: dict, X: np.ndarray, t: np.ndarray) -> dict:
    """d loss / d parameter for every parameter (chain rule, FP64)."""
    y, (X, z1, a1, z2, a2) = forward(P, X)
    B = X.shape[0]
    dy = (2.0 / B) * (y - t)[:, None]          # [B][1]
    g = {"W3": a2.T @ dy, "b3": dy.sum(0)}
    da2 = dy @ P["W3"].T
    dz2 = da2 * (z2 > 0)
    g["W2"] = a1.T @ dz2
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ P["W2"].T
    dz1 = da1 * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(P: dict, G: dict, state: dict, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; `step` counts from 1."""
    for k in PARAMS:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1 - beta1) * G[k]
        v[...] = beta2 * v + (1 - beta2) * G[k] ** 2
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
