"""FP64 oracle of the cost-model MLP (test infrastructure only).

The paper has no learned component (it tunes unroll factors empirically and
always fuses everything, §VII-C); the cost model is an addition of this
project. Its definition here is the textbook one:

  h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3
  loss = mean over rows of (y - t)^2
  Adam (Kingma & Ba, 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Shapes: X [N, F], W1 [H, F], b1 [H], W2 [H, H], b2 [H], W3 [1, H], b3 [1].
Gradients are derived by hand (chain rule), with relu'(0) = 0.
"""

from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def forward(p: dict, X: np.ndarray):
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y[:, 0], {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def loss(y: np.ndarray, t: np.ndarray) -> float:
    r = y - np.asarray(t, np.float64)
    return float(np.mean(r * r))


def backward(p: dict, cache: dict, y: np.ndarray, t: np.ndarray) -> dict:
    n = y.shape[0]
    dy = (2.0 / n) * (y - np.asarray(t, np.float64))          # d loss / d y, [N]
    g = {}
    g["W3"] = dy[None, :] @ cache["h2"]                       # [1, H]
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] @ p["W3"]                               # [N, H]
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; ``step`` counts from 1."""
    for k in PARAM_NAMES:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mhat = m[k] / (1.0 - beta1 ** step)
        vhat = v[k] / (1.0 - beta2 ** step)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v
