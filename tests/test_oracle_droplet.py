"""Pins of the oracle's largest-droplet search and droplet theory (Sec. 3).

The cluster search is checked against networkx's connected components of
its own periodic grid graph (a library routine that shares nothing with the
oracle) and against configurations whose largest droplet is known by
construction.  The brute-force lambda(Delta) is checked against the critical
values the paper prints (tests/golden/droplet_critical.txt) and against
properties of Eqs. 8-10 that hold for any parameters.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import chain, droplet

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _critical():
    rows = []
    for line in open(os.path.join(GOLDEN, "droplet_critical.txt")):
        if line.strip() and not line.startswith("#"):
            d, dc, lc = line.split()
            rows.append((int(d), float(dc), float(Fraction(lc))))
    return rows


def _nx_largest(d, L, occ):
    nx = pytest.importorskip("networkx")
    g = nx.grid_graph(dim=[L] * d, periodic=True)
    keep = [t for t in g.nodes if occ[sum(int(t[k]) * L ** k for k in range(d))]]
    sub = g.subgraph(keep)
    return max((len(c) for c in nx.connected_components(sub)), default=0)


@pytest.mark.parametrize("d,L", [(2, 3), (2, 4), (2, 7), (2, 12), (3, 3), (3, 4), (3, 6)])
def test_largest_droplet_matches_networkx(d, L):
    rng = np.random.default_rng(100 * d + L)
    V = L ** d
    for rho in (0.1, 0.3, 0.5, 0.7):
        for _ in range(4):
            occ = (rng.random(V) < rho).astype(np.uint8)
            assert chain.largest_droplet(d, L, occ) == _nx_largest(d, L, occ)


def test_largest_droplet_constructed_cases():
    L = 8
    z = np.zeros((L, L), np.uint8)
    assert chain.largest_droplet(2, L, z) == 0
    assert chain.largest_droplet(2, L, np.ones((L, L), np.uint8)) == L * L
    cb = (np.add.outer(np.arange(L), np.arange(L)) % 2).astype(np.uint8)
    assert chain.largest_droplet(2, L, cb) == 1               # no two particles touch
    row = z.copy()
    row[3, :] = 1                                             # wraps around the boundary
    assert chain.largest_droplet(2, L, row) == L
    blocks = z.copy()
    blocks[0:2, 0:2] = 1                                      # 4 particles
    blocks[4:6, 4:7] = 1                                      # 6 particles, not touching
    assert chain.largest_droplet(2, L, blocks) == 6
    corner = z.copy()
    corner[0, 0] = corner[0, L - 1] = corner[L - 1, 0] = 1    # joined only through the wrap
    assert chain.largest_droplet(2, L, corner) == 3
    diag = z.copy()
    diag[2, 2] = diag[3, 3] = 1                               # diagonal is not a bond
    assert chain.largest_droplet(2, L, diag) == 1
    plane = np.zeros((5, 5, 5), np.uint8)
    plane[:, :, 2] = 1
    assert chain.largest_droplet(3, 5, plane) == 25


@pytest.mark.parametrize("d,delta_c,lambda_c", _critical())
def test_lambda_jumps_at_printed_critical_point(d, delta_c, lambda_c):
    """Below the printed Delta_c the minimiser is 0; just above it jumps to the
    printed lambda_c.  The printed Delta_c has four decimals, so the check is
    made 2e-4 away on either side."""
    assert droplet.lambda_of_delta(d, delta_c - 2e-4) == 0.0
    lam = droplet.lambda_of_delta(d, delta_c + 2e-4)
    assert lam == pytest.approx(lambda_c, abs=2e-3)
    # at the printed point both minima are (to its four decimals) equal
    f0 = droplet.free_energy_bracket(d, delta_c, 0.0)
    fc = droplet.free_energy_bracket(d, delta_c, lambda_c)
    assert abs(float(fc) - float(f0)) < 1e-4


def test_lambda_limits_and_monotonicity():
    for d in (2, 3):
        assert droplet.lambda_of_delta(d, 0.0) == 0.0
        prev = 0.0
        for D in np.linspace(0.0, 20.0, 41):
            lam = droplet.lambda_of_delta(d, D, points=200_001)
            assert lam >= prev - 1e-5          # more excess never shrinks the droplet
            prev = lam
        # Delta -> infinity: the whole excess sits in the droplet
        assert droplet.lambda_of_delta(d, 1e6) > 0.999


def test_delta_properties():
    # no excess over the background: V_L = 0, Delta = 0
    assert droplet.excess_volume(1000, 10.0, 0.01) == pytest.approx(0.0, abs=1e-12)
    assert droplet.delta(2, 1000, 10.0, 0.01, 0.03, 1.0) == 0.0
    # without background (rho0 = 0) the whole excess is N
    assert droplet.excess_volume(900, 50, 0.0) == 50
    # fixed density: Delta grows like V^(1/d) (V_L^((d+1)/d) / V with V_L ~ V)
    for d in (2, 3):
        a = droplet.delta(d, 10 ** 4, 500, 0.005, 0.02, 1.1)
        b = droplet.delta(d, 8 * 10 ** 4, 4000, 0.005, 0.02, 1.1)
        assert b / a == pytest.approx(8 ** (1 / d), rel=1e-12)
    # Delta is inversely proportional to kappa_hat and to tau_W
    a = droplet.delta(3, 27000, 300, 0.0027, 0.006, 2.861)
    assert droplet.delta(3, 27000, 300, 0.0027, 0.012, 2.861) == pytest.approx(a / 2, rel=1e-12)
    assert droplet.delta(3, 27000, 300, 0.0027, 0.006, 2 * 2.861) == pytest.approx(a / 2, rel=1e-12)
    assert math.isfinite(a) and a > 0
