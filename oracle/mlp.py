"""Reference of the cost model network: 16 -> 64 -> 64 -> 1, ReLU, mean squared error.

Test infrastructure only (see oracle/__init__.py).  Plain float64 numpy, written from the
definition of a fully connected network and of its gradient by the chain rule; pinned in
tests/test_oracle_mlp.py by central finite differences and by closed forms.

Parameter vector layout (5313 values): W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3.
Features are standardized as (x - mean) / std before the first layer.
"""

from __future__ import annotations

import numpy as np

F, H = 16, 64
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", ())]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape) if shape else p[o]
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X, mean=None, std=None):
    """Returns (y, cache) for rows of X."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    x = (X - (0 if mean is None else mean)) / (1 if std is None else std)
    a1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0)
    y = h2 @ w["W3"] + w["b3"]
    return y, (x, a1, h1, a2, h2)


def loss(p, X, y, mean=None, std=None):
    f, _ = forward(p, X, mean, std)
    return float(np.mean((f - np.asarray(y, dtype=np.float64)) ** 2))


def gradient(p, X, y, mean=None, std=None):
    """d loss / d p by the chain rule, in the packed layout."""
    w = unpack(p)
    f, (x, a1, h1, a2, h2) = forward(p, X, mean, std)
    n = x.shape[0]
    d = 2.0 * (f - np.asarray(y, dtype=np.float64)) / n  # d loss / d f
    g = {"W3": h2.T @ d, "b3": d.sum()}
    d2 = np.outer(d, w["W3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return pack(g)
