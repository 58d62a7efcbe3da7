"""Pins of the float64 seeding network: central finite differences of the loss
against the backward pass, and GELU's textbook values."""
import math

import numpy as np

from oracle import mlp


def test_gelu_textbook_values():
    z = np.array([0.0, 1.0, -1.0, 6.0, -6.0])
    g = mlp.gelu(z)
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15          # Phi(1)
    assert abs(g[2] + 0.15865525393145707) < 1e-15         # -Phi(-1)
    assert abs(g[3] - 6.0) < 1e-8 and abs(g[4]) < 1e-8
    # derivative against a central difference
    h = 1e-6
    zz = np.linspace(-4, 4, 33)
    fd = (mlp.gelu(zz + h) - mlp.gelu(zz - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(zz), fd, atol=1e-8)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = mlp.init_params(rng, hidden=16)
    X = rng.normal(size=(12, 4))
    t = rng.normal(size=12)
    g = mlp.backward(params, X, t)
    h = 1e-6
    for name, p in params.items():
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(params, X, t)
            flat[i] = old - h
            lm = mlp.loss(params, X, t)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)


def test_forward_linear_limit():
    """Large positive pre-activations make GELU the identity: the network is
    then the plain product of its affine maps."""
    rng = np.random.default_rng(1)
    params = mlp.init_params(rng, hidden=8)
    params["b1"][:] = 50.0
    params["b2"][:] = 50.0
    params["W2"] = np.abs(params["W2"]) * 0.01
    X = rng.normal(size=(5, 4)) * 0.1
    y, _ = mlp.forward(params, X)
    h1 = X @ params["W1"].T + params["b1"]
    h2 = h1 @ params["W2"].T + params["b2"]
    lin = (h2 @ params["W3"].T + params["b3"])[:, 0]
    np.testing.assert_allclose(y, lin, rtol=1e-12, atol=1e-9)
    assert math.isfinite(float(y.sum()))
