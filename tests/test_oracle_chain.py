"""Pins of the oracle's acceptance thresholds and Markov chain (Sec. 2).

The chain is checked against exact statistical mechanics on lattices small
enough to enumerate: detailed balance of the exact transition matrix with
respect to pi(x) ~ W(E(x)), stationary energy histograms H(E) ~ Omega(E) W(E)
from long runs, the infinite-temperature and canonical special cases, and
state invariants.
"""
import math

import numpy as np
import pytest

from oracle import chain, muca

U32MAX = 0xFFFFFFFF


# ---------------------------------------------------------------- thresholds --

def test_thresholds_flat_weights_accept_everything_in_window():
    d, e_lo, e_hi = 2, -10, 0
    T = chain.thresholds(d, e_lo, e_hi, np.zeros(11))
    for b in range(11):
        for j, de in enumerate(range(-2 * d, 2 * d + 1)):
            inside = 0 <= b + de <= 10
            assert T[b, j] == (U32MAX if inside else 0)


def test_thresholds_approximate_metropolis_ratio():
    """T/2^32 lies within 2^-32 below min(1, W(E_n)/W(E_o)) for every entry."""
    rng = np.random.default_rng(3)
    d, e_lo, e_hi = 3, -40, 0
    lnW = rng.normal(scale=3.0, size=41)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    for b in range(41):
        for j, de in enumerate(range(-2 * d, 2 * d + 1)):
            if not 0 <= b + de <= 40:
                assert T[b, j] == 0
                continue
            p = min(1.0, math.exp(lnW[b + de] - lnW[b]))
            if T[b, j] == U32MAX:
                assert p == 1.0
            else:
                q = int(T[b, j]) / 2.0 ** 32
                assert p - 2.0 ** -31 <= q <= p


def test_thresholds_canonical_closed_form():
    """lnW = -beta E: T(dE) = floor(2^32 e^{-beta dE}) for dE > 0, all-accept otherwise."""
    beta = 0.7
    e_lo, e_hi = -20, 0
    lnW = np.array([-beta * e for e in range(e_lo, e_hi + 1)])
    T = chain.thresholds(2, e_lo, e_hi, lnW)
    for b in range(4, 17):
        for j, de in enumerate(range(-4, 5)):
            if de <= 0:
                assert T[b, j] == U32MAX
            else:
                exact = math.exp(-beta * de) * 2.0 ** 32
                assert abs(int(T[b, j]) - exact) <= 1.0 + 1e-6 * exact


# -------------------------------------------------------- detailed balance ---

@pytest.mark.parametrize("N", [3, 4])
def test_exact_transition_matrix_detailed_balance(N):
    """3x3 lattice, random weights: pi P = pi with pi(x) ~ exp(lnW(E(x)))."""
    d, L = 2, 3
    rng = np.random.default_rng(N)
    e_lo, e_hi = -d * N, 0
    lnW = rng.normal(scale=1.5, size=e_hi - e_lo + 1)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    states, en, P = muca.transition_matrix(d, L, N, T, e_lo)
    assert len(states) == math.comb(9, N)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    pi = np.exp(lnW[en - e_lo])
    pi /= pi.sum()
    assert np.abs(pi @ P - pi).max() < 1e-9
    # pairwise balance up to the 2^-32 threshold quantisation
    flow = pi[:, None] * P
    off = ~np.eye(len(states), dtype=bool)
    scale = np.maximum(flow, flow.T)[off]
    diff = np.abs(flow - flow.T)[off]
    assert (diff <= 2.0 ** -31 * pi.max() + 1e-15 + 1e-12 * scale).all()


# ------------------------------------------------------------ long chains ----

def _run_hist(d, L, N, lnW, e_lo, e_hi, walkers, sweeps, seed):
    S, occ, E = chain.init_walkers(d, L, N, walkers, seed)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    hist, acc = chain.run_walkers(d, L, N, seed, 0, sweeps * N, e_lo, e_hi, T, S, occ, E)
    return hist, acc, (S, occ, E)


def test_infinite_temperature_histogram_is_omega():
    """lnW = 0: every move accepted, H(E)/sum H -> Omega(E)/C(V,N)."""
    d, L, N = 2, 4, 8
    om = chain.enumerate_omega(d, L, N)
    hist, acc, _ = _run_hist(d, L, N, np.zeros(17), -16, 0, 32, 20000, 5)
    assert acc.sum() == 32 * 20000 * N
    H = hist.sum(axis=0)
    n = H.sum()
    tot = math.comb(16, 8)
    for e in range(-16, 1):
        p = om.get(e, 0) / tot
        if p == 0:
            assert H[e + 16] == 0
        else:
            assert abs(H[e + 16] / n - p) < 6 * math.sqrt(p * (1 - p) / n) * 4 + 1e-4


def test_multicanonical_stationary_histogram_3x3():
    """Random lnW on 3x3, N=4: H(E) ~ Omega(E) W(E) (chi-square over energies)."""
    d, L, N = 2, 3, 4
    om = chain.enumerate_omega(d, L, N)
    rng = np.random.default_rng(11)
    lnW = rng.normal(scale=1.0, size=9)
    hist, _, _ = _run_hist(d, L, N, lnW, -8, 0, 16, 40000, 17)
    # walker-level means give an error bar that includes autocorrelation
    fr = hist / hist.sum(axis=1, keepdims=True)
    mean = fr.mean(axis=0)
    sem = fr.std(axis=0, ddof=1) / math.sqrt(fr.shape[0])
    z = 0.0
    for e, c in om.items():
        p = c * math.exp(lnW[e + 8]) / sum(cc * math.exp(lnW[ee + 8]) for ee, cc in om.items())
        assert abs(mean[e + 8] - p) < 5 * sem[e + 8] + 1e-5
        z += ((mean[e + 8] - p) / max(sem[e + 8], 1e-9)) ** 2
    assert z < len(om) + 6 * math.sqrt(2 * len(om))


def test_canonical_special_case_mean_energy():
    """lnW = -beta E turns the method into canonical Metropolis: <E>_beta exact."""
    d, L, N = 2, 4, 8
    om = chain.enumerate_omega(d, L, N)
    beta = 0.8
    lnW = np.array([-beta * e for e in range(-16, 1)])
    hist, _, _ = _run_hist(d, L, N, lnW, -16, 0, 16, 30000, 23)
    per_walker = (hist * np.arange(-16, 1)[None, :]).sum(axis=1) / hist.sum(axis=1)
    exact = muca.exact_mean_energy(om, beta)
    sem = per_walker.std(ddof=1) / math.sqrt(len(per_walker))
    assert abs(per_walker.mean() - exact) < 5 * sem + 1e-3


@pytest.mark.parametrize("d,L,N", [(2, 16, 32), (3, 6, 30)])
def test_state_invariants_after_runs(d, L, N):
    rng = np.random.default_rng(1)
    e_lo = -d * N
    lnW = np.cumsum(rng.normal(scale=0.3, size=d * N + 1))
    hist, acc, (S, occ, E) = _run_hist(d, L, N, lnW, e_lo, 0, 8, 50, 99)
    V = L ** d
    assert (hist.sum(axis=1) == 50 * N).all()
    for w in range(8):
        assert sorted(S[w].tolist()) == list(range(V))
        assert occ[w].sum() == N
        assert set(np.nonzero(occ[w])[0].tolist()) == set(S[w, :N].tolist())
        assert E[w] == chain.energy(d, L, occ[w])
    assert (acc > 0).all()


def test_state_carries_over_between_iterations():
    """Two iterations in sequence equal one walker run twice with iteration tags 0, 1."""
    d, L, N = 2, 8, 10
    lnW = np.zeros(21)
    T = chain.thresholds(d, -20, 0, lnW)
    S, occ, E = chain.init_walkers(d, L, N, 4, 42)
    h0, _ = chain.run_walkers(d, L, N, 42, 0, 100, -20, 0, T, S, occ, E)
    h1, _ = chain.run_walkers(d, L, N, 42, 1, 100, -20, 0, T, S, occ, E)
    S2, occ2, E2 = chain.init_walkers(d, L, N, 4, 42)
    g0, _ = chain.run_walkers(d, L, N, 42, 0, 100, -20, 0, T, S2, occ2, E2)
    np.testing.assert_array_equal(h0, g0)
    g1, _ = chain.run_walkers(d, L, N, 42, 1, 100, -20, 0, T, S2, occ2, E2)
    np.testing.assert_array_equal(h1, g1)
    np.testing.assert_array_equal(S, S2)
    # a different iteration tag gives a different trajectory
    S3, occ3, E3 = chain.init_walkers(d, L, N, 4, 42)
    g2, _ = chain.run_walkers(d, L, N, 42, 7, 100, -20, 0, T, S3, occ3, E3)
    assert not np.array_equal(S3, S2) or not np.array_equal(g2, h0)


def test_subset_walkers_match_full_run():
    """Walker w of a batch equals walker w run alone (independent chains, Sec. 2)."""
    d, L, N = 2, 16, 32
    T = chain.thresholds(d, -64, 0, np.zeros(65))
    S, occ, E = chain.init_walkers(d, L, N, 10, 3)
    h, _ = chain.run_walkers(d, L, N, 3, 5, 500, -64, 0, T, S, occ, E)
    pick = [2, 7]
    S1, occ1, E1 = chain.init_walkers(d, L, N, 10, 3)
    S1, occ1, E1 = S1[pick].copy(), occ1[pick].copy(), E1[pick].copy()
    h1, _ = chain.run_walkers(d, L, N, 3, 5, 500, -64, 0, T, S1, occ1, E1, walkers=pick)
    np.testing.assert_array_equal(h1, h[pick])
    np.testing.assert_array_equal(S1, S[pick])


def test_fixed_magnetisation_ising_matches_enumeration_through_eq5():
    """Sec. 4 cross-check: micromagnetic Ising at beta^I versus the exact gas
    density of states mapped by Eq. 5 (beta = 4 beta^I, H_I = 4 (E - c))."""
    d, L, N = 2, 4, 8
    om = chain.enumerate_omega(d, L, N)
    beta_i = 0.369
    c = muca.ising_constant(d, L, N)
    exact_gas = muca.exact_mean_energy(om, 4 * beta_i)
    exact_ising = 4.0 * (exact_gas - c)
    vals = [chain.ising_fixed_m(d, L, N, s, beta_i, 200000, 2000)[0] for s in range(8)]
    sem = np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - exact_ising) < 5 * sem + 0.02
