"""FP64 reference of the surrogate network and its gradients.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network (fixed architecture): x in R^5 -> a1 = W1 x + b1 (128) -> h1 = gelu(a1)
-> a2 = W2 h1 + b2 (128) -> h2 = gelu(a2) -> y = W3 h2 + b3 (12), with the exact
gelu(a) = a Phi(a), Phi the standard normal CDF.  Loss over a batch of n
samples: L = sum((y - t)^2) / (12 n).

Written from the definitions (chain rule); pinned by a central-difference
test, not by another implementation.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SHAPES = {"W1": (128, 5), "b1": (128,), "W2": (128, 128), "b2": (128,), "W3": (12, 128),
          "b3": (12,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())  # 18,828


def gelu(a):
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    # d/da [a Phi(a)] = Phi(a) + a phi(a)
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2 * math.pi)


def unpack(flat):
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[k], np.float64).ravel() for k in ORDER])


def forward(p, x):
    """x: [n, 5] -> (y [n, 12], cache)."""
    a1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, a1, h1, a2, h2)


def loss_and_grad(p, x, t):
    """Mean-squared error and its gradient with respect to every parameter."""
    y, (x, a1, h1, a2, h2) = forward(p, x)
    n = x.shape[0]
    r = y - t
    L = float(np.sum(r * r) / (12 * n))
    dy = 2.0 * r / (12 * n)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    da2 = (dy @ p["W3"]) * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = (da2 @ p["W2"]) * gelu_grad(a1)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(0)
    return L, g
