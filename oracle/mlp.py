"""float64 reference of the weight-seeding network (test infrastructure only).

The network maps a 4-vector of features (built by the caller from
(d, L, rho, E/V)) to a prediction of ln Omega(E)/V:

    h1 = gelu(W1 x + b1)      W1: [128, 4]
    h2 = gelu(W2 h1 + b2)     W2: [128, 128]
    y  = W3 h2 + b3           W3: [1, 128]

with gelu(z) = z * Phi(z) (Phi the standard normal CDF) and the loss
L = mean over the batch of (y - t)^2.  The weights given here are used as
they are; the tests pass the bf16-rounded values the GPU stores, so that only
the GPU's bf16 activations and fp32 accumulation differ from this reference.
The network is not part of the paper; it seeds lnW, after which the paper's
iteration (Sec. 2) runs unchanged.
"""
from __future__ import annotations

import math

import numpy as np

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(z: np.ndarray) -> np.ndarray:
    return np.vectorize(math.erf, otypes=[np.float64])(z)


def gelu(z: np.ndarray) -> np.ndarray:
    return 0.5 * z * (1.0 + _erf(z / _SQRT2))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    cdf = 0.5 * (1.0 + _erf(z / _SQRT2))
    pdf = _INV_SQRT_2PI * np.exp(-0.5 * z * z)
    return cdf + z * pdf


def forward(params: dict, X: np.ndarray):
    """Returns (y [B], cache) for X [B, 4]."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y[:, 0], (X, z1, h1, z2, h2)


def loss(params: dict, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(params, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(params: dict, X: np.ndarray, t: np.ndarray):
    """Gradients of the mean squared error by the chain rule, layer by layer."""
    y, (X, z1, h1, z2, h2) = forward(params, X)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B        # [B]
    g = {}
    g["W3"] = dy[None, :] @ h2                                   # [1, 128]
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] * params["W3"][0][None, :]                 # [B, 128]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return g


def init_params(rng: np.random.Generator, hidden: int = 128) -> dict:
    """Scaled-uniform initialisation (fan-in), float64."""
    def u(shape, fan_in):
        lim = 1.0 / math.sqrt(fan_in)
        return rng.uniform(-lim, lim, size=shape)
    return {
        "W1": u((hidden, 4), 4), "b1": u((hidden,), 4),
        "W2": u((hidden, hidden), hidden), "b2": u((hidden,), hidden),
        "W3": u((1, hidden), hidden), "b3": u((1,), hidden),
    }
