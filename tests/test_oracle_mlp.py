"""Pins of the FP64 MLP oracle: gradients against central finite differences,
a one-hidden-unit network computed by hand, Adam's first step, and three
Adam steps derived by hand (tests/golden/adam_three_steps.txt)."""

import os

import numpy as np

from oracle import mlp
from paper_2005_13014_gb300 import inputs


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = inputs.mlp_init(7, hidden=5, seed=3)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.uniform(-0.1, 0.1, p[k].shape)
    X = rng.normal(size=(9, 7))
    t = rng.normal(size=9)
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, t)
    eps = 1e-6
    for k in mlp.PARAM_NAMES:
        num = np.zeros_like(p[k])
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[k][idx]
            p[k][idx] = old + eps
            lp = mlp.loss(mlp.forward(p, X)[0], t)
            p[k][idx] = old - eps
            lm = mlp.loss(mlp.forward(p, X)[0], t)
            p[k][idx] = old
            num[idx] = (lp - lm) / (2 * eps)
        scale = max(np.max(np.abs(num)), 1e-12)
        assert np.max(np.abs(num - g[k])) <= 1e-6 * scale + 1e-10, k


def test_one_hidden_unit_by_hand():
    # x = [1, 2]; W1 = [[0.5, -0.25]] -> z1 = 0 + b1 = 0.25 -> h1 = 0.25
    # W2 = [[2]], b2 = -0.25 -> z2 = 0.25 -> h2 = 0.25; W3 = [[4]], b3 = 1 -> y = 2
    p = {"W1": np.array([[0.5, -0.25]]), "b1": np.array([0.25]), "W2": np.array([[2.0]]),
         "b2": np.array([-0.25]), "W3": np.array([[4.0]]), "b3": np.array([1.0])}
    y, cache = mlp.forward(p, np.array([[1.0, 2.0]]))
    assert y[0] == 2.0
    # t = 3: loss = 1, dy = -2; dW3 = -2*0.25 = -0.5; db3 = -2; dh2 = -8 -> dz2 = -8
    # dW2 = -8*0.25 = -2; db2 = -8; dh1 = -16 -> dz1 = -16; dW1 = [-16, -32]; db1 = -16
    g = mlp.backward(p, cache, y, np.array([3.0]))
    assert mlp.loss(y, np.array([3.0])) == 1.0
    assert g["W3"].tolist() == [[-0.5]] and g["b3"].tolist() == [-2.0]
    assert g["W2"].tolist() == [[-2.0]] and g["b2"].tolist() == [-8.0]
    assert g["W1"].tolist() == [[-16.0, -32.0]] and g["b1"].tolist() == [-16.0]


def test_adam_first_step_moves_by_lr():
    p = {k: np.array([1.0]) for k in mlp.PARAM_NAMES}
    g = {k: np.array([0.5 if i % 2 else -2.0]) for i, k in enumerate(mlp.PARAM_NAMES)}
    m = {k: np.zeros(1) for k in mlp.PARAM_NAMES}
    v = {k: np.zeros(1) for k in mlp.PARAM_NAMES}
    mlp.adam_step(p, g, m, v, 1, lr=0.01)
    for k in mlp.PARAM_NAMES:
        # bias-corrected first step: lr * g / (|g| + eps)
        want = 1.0 - 0.01 * g[k][0] / (abs(g[k][0]) + 1e-8)
        assert abs(p[k][0] - want) < 1e-15


def test_adam_three_steps_match_hand_derivation():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "adam_three_steps.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    assert len(rows) == 3
    p = {k: np.array([1.0]) for k in mlp.PARAM_NAMES}
    m = {k: np.zeros(1) for k in mlp.PARAM_NAMES}
    v = {k: np.zeros(1) for k in mlp.PARAM_NAMES}
    for step, grad, m_want, v_want, num, den in rows:
        g = {k: np.array([grad]) for k in mlp.PARAM_NAMES}
        mlp.adam_step(p, g, m, v, int(step), lr=0.5, beta1=0.5, beta2=0.75, eps=0.0)
        for k in mlp.PARAM_NAMES:
            assert m[k][0] == m_want and v[k][0] == v_want, (step, k)
            assert abs(p[k][0] - num / den) <= 1e-15, (step, k, p[k][0], num / den)
