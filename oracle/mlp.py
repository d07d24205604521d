"""FP64 oracle of the surrogate network that pre-screens EMPSO particles.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no
surrogate; this restates the network the library trains online: a
multilayer perceptron K -> H -> H -> 1 with ReLU hidden layers predicting the
standardised log-misfit of a particle from its control-node vector scaled to
[-1, 1], trained on the half mean squared error with Adam (Kingma & Ba 2015:
m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, w -= lr m_hat / (sqrt(v_hat) + eps)
with bias corrections 1 - b^t).

Parameters are kept as a dict of float64 arrays:
  W1 [H][K], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1].
Pins (tests/test_oracle_mlp.py): central finite differences of the loss,
the closed-form first Adam step, and the fit of a known function.
"""
from __future__ import annotations

import numpy as np

ORDER = ("W1", "b1", "W2", "b2", "w3", "b3")


def shapes(K: int, H: int) -> dict:
    return {"W1": (H, K), "b1": (H,), "W2": (H, H), "b2": (H,), "w3": (H,), "b3": (1,)}


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(v: np.ndarray, K: int, H: int) -> dict:
    out, o = {}, 0
    for k in ORDER:
        shp = shapes(K, H)[k]
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def forward(p: dict, X: np.ndarray):
    """y [B] and the activations (Z1, A1, Z2, A2) for backward."""
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    y = A2 @ p["w3"] + p["b3"][0]
    return y, (Z1, A1, Z2, A2)


def loss(p: dict, X: np.ndarray, t: np.ndarray) -> float:
    """L = 1/(2B) sum_b (y_b - t_b)^2."""
    y, _ = forward(p, X)
    r = y - np.asarray(t, dtype=np.float64)
    return 0.5 * float(np.mean(r * r))


def backward(p: dict, X: np.ndarray, t: np.ndarray):
    """Gradients of L with respect to every parameter (dict), and L."""
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    y, (Z1, A1, Z2, A2) = forward(p, X)
    r = y - np.asarray(t, dtype=np.float64)
    dy = r / B
    g = {"w3": A2.T @ dy, "b3": np.array([dy.sum()])}
    dZ2 = np.outer(dy, p["w3"]) * (Z2 > 0)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return g, 0.5 * float(np.mean(r * r))


class Adam:
    def __init__(self, p: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in p.items()}
        self.v = {k: np.zeros_like(v) for k, v in p.items()}
        self.t = 0

    def step(self, p: dict, g: dict) -> None:
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        for k in p:
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g[k]
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g[k] * g[k]
            p[k] -= self.lr * (self.m[k] / c1) / (np.sqrt(self.v[k] / c2) + self.eps)


def init_params(K: int, H: int, seed: int) -> dict:
    """He-uniform weights, zero biases (any initialisation works for the pins)."""
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in shapes(K, H).items():
        if k.startswith("b"):
            p[k] = np.zeros(shp)
        else:
            fan_in = shp[-1] if len(shp) == 2 else H
            lim = np.sqrt(6.0 / fan_in)
            p[k] = rng.uniform(-lim, lim, shp)
    return p


def to_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rnd = ((u >> 16) & 1) + 0x7FFF
    q = ((u + rnd) >> 16) << 16
    return q.astype(np.uint32).view(np.float32).astype(np.float64)
