"""Pins for the cost-model reference network (oracle/mlp.py): central finite differences of the
loss, and closed forms for degenerate parameters."""

import numpy as np
import pytest

from oracle import mlp


def rand_params(rng, scale=0.3):
    return rng.normal(0, scale, mlp.NPARAM)


@pytest.mark.parametrize("seed", range(4))
def test_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = rand_params(rng)
    X = rng.normal(0, 1, (9, mlp.F))
    y = rng.normal(0, 1, 9)
    g = mlp.gradient(p, X, y)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_closed_forms():
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, (5, mlp.F))
    y = rng.normal(0, 1, 5)
    w = mlp.unpack(np.zeros(mlp.NPARAM))
    w = {k: np.array(v, copy=True) for k, v in w.items()}
    w["b3"] = 0.7
    p = mlp.pack(w)
    f, _ = mlp.forward(p, X)
    assert np.allclose(f, 0.7)  # all hidden units dead: output is the last bias
    g = mlp.unpack(mlp.gradient(p, X, y))
    assert np.isclose(g["b3"], 2 * np.mean(0.7 - y))
    assert not np.any(g["W1"]) and not np.any(g["W2"]) and not np.any(g["W3"])
    # a single live path: relu(x0) * 1 * 1 with b1[0] = b2[0] = 0
    w2 = {k: np.zeros_like(np.asarray(v, dtype=float)) for k, v in w.items()}
    w2["W1"][0, 0] = 1.0
    w2["W2"][0, 0] = 1.0
    w2["W3"][0] = 1.0
    w2["b3"] = 0.0
    f2, _ = mlp.forward(mlp.pack(w2), X)
    assert np.allclose(f2, np.maximum(X[:, 0], 0))


def test_standardization_is_applied():
    rng = np.random.default_rng(3)
    p = rand_params(rng)
    X = rng.normal(5, 2, (7, mlp.F))
    mean, std = X.mean(0), X.std(0) + 0.1
    a, _ = mlp.forward(p, X, mean, std)
    b, _ = mlp.forward(p, (X - mean) / std)
    assert np.allclose(a, b)
