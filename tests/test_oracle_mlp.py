"""Pins of the FP64 surrogate-network reference against mathematics."""

import math

import numpy as np

from oracle import mlp


def random_params(rng, scale=0.3):
    return {k: rng.normal(0, scale, s) for k, s in mlp.SHAPES.items()}


def test_parameter_count_matches_architecture():
    assert mlp.N_PARAMS == 5 * 128 + 128 + 128 * 128 + 128 + 128 * 12 + 12 == 18828


def test_gelu_closed_forms():
    a = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in a]))
    assert np.allclose(mlp.gelu(a), a * phi, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(a), fd, atol=1e-9)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    p = random_params(rng)
    x = rng.normal(size=(7, 5))
    t = rng.normal(size=(7, 12))
    L, g = mlp.loss_and_grad(p, x, t)
    flat = mlp.pack(p)
    gflat = mlp.pack(g)
    idx = rng.choice(flat.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        Lp, _ = mlp.loss_and_grad(mlp.unpack(fp), x, t)
        Lm, _ = mlp.loss_and_grad(mlp.unpack(fm), x, t)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_linear_limit():
    """With W1 = W2 = 0 the hidden activations are gelu(b): the output is affine
    in those constants (a hand-computable case)."""
    rng = np.random.default_rng(4)
    p = random_params(rng)
    p["W1"][:] = 0
    p["W2"][:] = 0
    x = rng.normal(size=(3, 5))
    y, _ = mlp.forward(p, x)
    h2 = mlp.gelu(p["b2"])
    assert np.allclose(y, np.tile(p["W3"] @ h2 + p["b3"], (3, 1)), atol=1e-14)
