"""Pins of the oracle's replica exchange (parallel tempering, Sec. 3).

Exchanges with the acceptance min(1, exp((beta_k - beta_k+1)(E_k - E_k+1)))
leave the product of the canonical distributions invariant, so a tempering
ladder run with the oracle's canonical walkers must sample, at every
temperature, the canonical energy distribution Omega(E) exp(-beta E) of the
enumerated lattice (Eq. 1).  A wrong sign or a wrong pairing breaks that.
"""
import math

import numpy as np

from oracle import chain


def _ladder_histograms(d, L, N, betas, walkers, rounds, burn, attempts, exchange=True, seed0=1000):
    K = len(betas)
    V = L ** d
    seeds = np.array([seed0 * (k + 1) for k in range(K)], dtype=np.uint64)
    S = np.zeros((K, walkers, V), np.int32)
    occ = np.zeros((K, walkers, V), np.uint8)
    E = np.zeros((K, walkers), np.int64)
    for k in range(K):
        S[k], occ[k], E[k] = chain.init_walkers(d, L, N, walkers, int(seeds[k]))
    e_lo = -d * N
    nb = d * N + 1
    T = [chain.thresholds(d, e_lo, 0, -b * np.arange(e_lo, 1, dtype=np.float64)) for b in betas]
    hist = np.zeros((K, nb), np.int64)
    acc_total = np.zeros(K - 1, np.int64)
    for r in range(rounds):
        for k in range(K):
            chain.run_walkers(d, L, N, int(seeds[k]), r, attempts, e_lo, 0, T[k], S[k], occ[k], E[k])
        if exchange:
            acc_total += chain.replica_exchange(betas, seeds, r, r % 2, S, occ, E)
        if r >= burn:
            for k in range(K):
                hist[k] += np.bincount(E[k] - e_lo, minlength=nb)
    return hist, acc_total, (S, occ, E)


def _canonical(omega, beta, e_lo, nb):
    p = np.zeros(nb)
    mx = max(-beta * e for e in omega)
    for e, c in omega.items():
        p[e - e_lo] = c * math.exp(-beta * e - mx)
    return p / p.sum()


def test_tempering_ladder_samples_canonical_marginals():
    d, L, N = 2, 4, 5
    betas = [0.2, 0.9, 1.8, 3.0]
    omega = chain.enumerate_omega(d, L, N)
    hist, acc, (S, occ, E) = _ladder_histograms(d, L, N, betas, walkers=256, rounds=1500, burn=100,
                                               attempts=1)
    assert (acc > 0).all()
    for k, b in enumerate(betas):
        p = hist[k] / hist[k].sum()
        q = _canonical(omega, b, -d * N, d * N + 1)
        assert 0.5 * np.abs(p - q).sum() < 0.03, (b, p.round(3), q.round(3))
    # configurations stay consistent after many exchanges
    for k in range(len(betas)):
        for w in range(0, 256, 37):
            assert occ[k, w].sum() == N and set(S[k, w, :N]) == set(np.nonzero(occ[k, w])[0])
            assert chain.energy(d, L, occ[k, w]) == E[k, w]


def test_equal_temperatures_always_exchange():
    d, L, N, W = 2, 5, 6, 16
    V = L ** d
    K = 3
    seeds = np.array([7, 70, 700], dtype=np.uint64)
    S = np.zeros((K, W, V), np.int32)
    occ = np.zeros((K, W, V), np.uint8)
    E = np.zeros((K, W), np.int64)
    for k in range(K):
        S[k], occ[k], E[k] = chain.init_walkers(d, L, N, W, int(seeds[k]))
    S0, E0 = S.copy(), E.copy()
    acc = chain.replica_exchange([1.0, 1.0, 1.0], seeds, 0, 0, S, occ, E)
    assert acc.tolist() == [W, 0]
    np.testing.assert_array_equal(S[0], S0[1])
    np.testing.assert_array_equal(S[1], S0[0])
    np.testing.assert_array_equal(S[2], S0[2])
    np.testing.assert_array_equal(E[:2], E0[[1, 0]])
    acc = chain.replica_exchange([1.0, 1.0, 1.0], seeds, 1, 1, S, occ, E)
    assert acc.tolist() == [0, W]


def test_exchange_acceptance_rate_matches_probability():
    """Many exchange proposals between two fixed energies: the accepted
    fraction estimates exp((beta_0 - beta_1)(E_0 - E_1)) within its binomial
    error."""
    d, L, N, W = 2, 6, 8, 4096
    V = L ** d
    seeds = np.array([11, 2222], dtype=np.uint64)
    S = np.zeros((2, W, V), np.int32)
    occ = np.zeros((2, W, V), np.uint8)
    E = np.zeros((2, W), np.int64)
    E[0] = -1
    E[1] = -6          # colder replica 0 holds the higher energy: exponent < 0 for beta_0 < beta_1
    betas = [0.5, 0.8]
    p = math.exp((betas[0] - betas[1]) * (E[0, 0] - E[1, 0]))
    total = 0
    n = 0
    for r in range(8):
        E[0] = -1
        E[1] = -6
        total += int(chain.replica_exchange(betas, seeds, r, 0, S, occ, E)[0])
        n += W
    rate = total / n
    assert abs(rate - p) < 5 * math.sqrt(p * (1 - p) / n), (rate, p)
