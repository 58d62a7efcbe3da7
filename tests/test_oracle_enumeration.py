"""Pins of the exact density of states Omega(E) (the W = 1/Omega target of Sec. 2).

The oracle's enumerator is checked against a brute force written here
(itertools over subsets, numpy.roll energies), against closed forms for two
and three particles, and against configurations counted by hand.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import chain


def _brute_omega(d, L, N):
    V = L ** d
    out = {}
    for combo in itertools.combinations(range(V), N):
        g = np.zeros(V, dtype=np.int64)
        g[list(combo)] = 1
        g = g.reshape((L,) * d)
        e = -int(sum((g * np.roll(g, 1, axis=ax)).sum() for ax in range(d)))
        out[e] = out.get(e, 0) + 1
    return out


@pytest.mark.parametrize("d,L,N", [(2, 3, 3), (2, 3, 4), (2, 4, 4), (2, 4, 8), (3, 3, 3)])
def test_enumeration_matches_brute_force(d, L, N):
    assert chain.enumerate_omega(d, L, N) == _brute_omega(d, L, N)


@pytest.mark.parametrize("d,L,N", [(2, 4, 8), (2, 5, 6), (3, 4, 3)])
def test_enumeration_total_is_binomial(d, L, N):
    assert sum(chain.enumerate_omega(d, L, N).values()) == math.comb(L ** d, N)


def test_4x4_n8_hand_counted_extremes_and_gaps():
    om = chain.enumerate_omega(2, 4, 8)
    # ground state: a 2x4 band wrapping the torus, 4 rows-pairs x 2 orientations
    assert om[-12] == 8
    # no bond: the two checkerboards
    assert om[0] == 2
    # impossible energies (gaps) of this system
    for e in (-11, -2, -1):
        assert e not in om


@pytest.mark.parametrize("d,L", [(2, 4), (2, 5), (3, 4)])
def test_closed_forms_two_and_three_particles(d, L):
    """N=2: Omega(-1) = dV (bonds), Omega(0) = C(V,2) - dV.
    N=3 (L >= 4): Omega(-2) = V C(2d,2) (paths of length two centred on a site),
    Omega(-1) = dV (V - 4d) (a bond plus a site off its closed neighbourhood),
    no triangles on the square/cubic lattice, so Omega(-3) = 0."""
    V = L ** d
    om2 = chain.enumerate_omega(d, L, 2)
    assert om2 == {-1: d * V, 0: math.comb(V, 2) - d * V}
    om3 = chain.enumerate_omega(d, L, 3)
    assert om3.get(-3, 0) == 0
    assert om3[-2] == V * math.comb(2 * d, 2)
    assert om3[-1] == d * V * (V - 4 * d)
    assert om3[0] == math.comb(V, 3) - om3[-2] - om3[-1]
