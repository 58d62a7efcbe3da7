"""Droplet theory of Sec. 3 (Eqs. 8-10), plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring).

lambda(Delta) is found by brute force: the bracket of Eq. 9,
f(lambda) = lambda^((d-1)/d) + Delta (1 - lambda)^2, is evaluated on a dense
uniform grid of [0, 1] and its smallest value taken; no calculus, no root
finding.
"""
from __future__ import annotations

import numpy as np


def excess_volume(V, N, rho0):
    """V_L = (N - N_0) / (1 - 2 rho0) with N_0 = rho0 V (Eq. 8)."""
    return (N - rho0 * V) / (1.0 - 2.0 * rho0)


def delta(d, V, N, rho0, kappa_hat, tau_W):
    """Delta of Eq. 10; 0 where there is no excess (V_L <= 0)."""
    vl = excess_volume(V, N, rho0)
    if vl <= 0:
        return 0.0
    return (1.0 - 2.0 * rho0) ** 2 / (2.0 * kappa_hat * tau_W) * vl ** ((d + 1) / d) / V


def free_energy_bracket(d, Delta, lam):
    lam = np.asarray(lam, dtype=np.float64)
    return lam ** ((d - 1) / d) + Delta * (1.0 - lam) ** 2


def lambda_of_delta(d, Delta, points=2_000_001):
    """Global minimiser of the Eq. 9 bracket over a uniform grid of [0, 1]."""
    lam = np.linspace(0.0, 1.0, points)
    f = free_energy_bracket(d, Delta, lam)
    return float(lam[int(np.argmin(f))])
