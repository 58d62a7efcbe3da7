"""Pins of the oracle's weight iteration, flatness and ln Omega (Sec. 2).

With exact histograms H ~ Omega W (what infinite statistics would give), the
simple iteration W/H must land on W = 1/Omega in one step, the recursion must
start as the simple iteration, keep the ideal weights fixed, and move each
log-ratio the fraction kappa of the way to its ideal value.  The full
multicanonical run must recover ln Omega of an enumerated lattice.
"""
import math

import numpy as np
import pytest

from oracle import chain, muca
from oracle.recursion import flatness, ln_omega, normalise, recursive_update, simple_update


def _exact_hist(om, lnW, e_lo, total=1e7):
    """H(E) = total * Omega(E) W(E) / Z, float64, zero where Omega = 0."""
    n = len(lnW)
    logs = {b: math.log(om[e_lo + b]) + lnW[b] for b in range(n) if (e_lo + b) in om}
    mx = max(logs.values())
    z = sum(math.exp(v - mx) for v in logs.values())
    H = np.zeros(n)
    for b, v in logs.items():
        H[b] = total * math.exp(v - mx) / z
    return H


def _ideal(om, e_lo, n):
    return np.array([-math.log(om[e_lo + b]) if (e_lo + b) in om else np.nan for b in range(n)])


def _agree_up_to_constant(a, b, mask, tol):
    diff = (a - b)[mask]
    assert np.ptp(diff) < tol


OM = chain.enumerate_omega(2, 4, 8)
E_LO = -16
NB = 17


def test_simple_update_reaches_inverse_omega_in_one_step():
    rng = np.random.default_rng(0)
    lnW = rng.normal(size=NB)
    H = _exact_hist(OM, lnW, E_LO)
    new = simple_update(lnW, H)
    mask = H > 0
    _agree_up_to_constant(new, _ideal(OM, E_LO, NB), mask, 1e-9)
    assert new.max() == 0.0
    # unvisited bins keep their weight (relative to the normalisation shift)
    shift = new[~mask] - lnW[~mask]
    assert np.ptp(shift) < 1e-12


def test_recursion_first_step_equals_simple_on_visited():
    rng = np.random.default_rng(1)
    lnW = rng.normal(size=NB)
    H = np.where(rng.random(NB) < 0.7, rng.integers(1, 1000, NB), 0).astype(np.float64)
    new_r, s_cum, phat = recursive_update(lnW, H, np.zeros(NB, bool), np.zeros(NB))
    new_s = simple_update(lnW, H)
    mask = H > 0
    _agree_up_to_constant(new_r, new_s, mask, 1e-10)
    np.testing.assert_array_equal(s_cum, mask)


def test_recursion_with_gaps_converges_and_stays_fixed():
    """4x4, N=8 has impossible energies (-11, -2, -1): pairs skip them."""
    lnW = np.zeros(NB)
    s_cum = np.zeros(NB, bool)
    phat = np.zeros(NB)
    for _ in range(3):
        H = _exact_hist(OM, lnW, E_LO)
        lnW, s_cum, phat = recursive_update(lnW, H, s_cum, phat)
    ideal = _ideal(OM, E_LO, NB)
    mask = s_cum.copy()
    _agree_up_to_constant(lnW, ideal, mask, 1e-9)
    H = _exact_hist(OM, lnW, E_LO)
    assert flatness(H, s_cum) > 1 - 1e-9


def test_flat_histogram_is_a_fixed_point():
    rng = np.random.default_rng(2)
    lnW = normalise(rng.normal(size=NB))
    H = np.full(NB, 5000.0)
    for _ in range(3):
        new, s_cum, phat = recursive_update(lnW, H, np.ones(NB, bool), np.ones(NB))
        np.testing.assert_allclose(new, lnW, atol=1e-12)


def test_recursion_moves_kappa_of_the_way():
    """Second step with exact data: ln R <- (1 - kappa) ln R + kappa ln R_ideal,
    kappa = g2 / (g1 + g2), the statistical weight of the new data."""
    lnW0 = np.zeros(NB)
    H1 = _exact_hist(OM, lnW0, E_LO, total=1e5)
    H1 *= np.linspace(0.5, 1.5, NB)           # a noisy first estimate
    lnW1, s1, p1 = recursive_update(lnW0, H1, np.zeros(NB, bool), np.zeros(NB))
    H2 = _exact_hist(OM, lnW1, E_LO, total=3e5)
    lnW2, s2, p2 = recursive_update(lnW1, H2, s1, p1)
    members = np.nonzero(s2)[0]
    ideal = _ideal(OM, E_LO, NB)
    for lo, hi in zip(members[:-1], members[1:]):
        g1 = H1[lo] * H1[hi] / (H1[lo] + H1[hi])
        g2 = H2[lo] * H2[hi] / (H2[lo] + H2[hi])
        kappa = g2 / (g1 + g2)
        r1 = lnW1[hi] - lnW1[lo]
        r_ideal = ideal[hi] - ideal[lo]
        r2 = lnW2[hi] - lnW2[lo]
        assert r2 == pytest.approx((1 - kappa) * r1 + kappa * r_ideal, abs=1e-9)


def test_unvisited_bins_follow_nearest_member_above():
    lnW = np.arange(NB, dtype=float) * 0.1
    H = np.zeros(NB)
    H[5] = 10
    H[6] = 20
    new, s_cum, _ = recursive_update(lnW, H, np.zeros(NB, bool), np.zeros(NB))
    # bins 0..4 move with bin 5, bins 7.. move with bin 6 (the top member)
    np.testing.assert_allclose(np.diff(new[:6]), np.diff(lnW[:6]), atol=1e-12)
    np.testing.assert_allclose(np.diff(new[6:]), np.diff(lnW[6:]), atol=1e-12)
    assert (new[6] - new[5]) == pytest.approx(0.1 + math.log(10) - math.log(20), abs=1e-12)


def test_flatness_definition_cases():
    s = np.array([False, True, True, True, False])
    H = np.array([0, 10, 5, 8, 0])
    assert flatness(H, s) == pytest.approx(0.5)
    assert flatness(H, s, 0, 3) == -1.0        # target end not visited
    assert flatness(np.array([0, 10, 0, 8, 0]), s) == 0.0


def test_ln_omega_exact_from_exact_histogram():
    rng = np.random.default_rng(4)
    lnW = rng.normal(size=NB)
    H = _exact_hist(OM, lnW, E_LO)
    est = ln_omega(lnW, H, 16, 8)
    for e, c in OM.items():
        assert est[e - E_LO] == pytest.approx(math.log(c), abs=1e-9)
    assert np.isnan(est[-11 - E_LO])


@pytest.mark.slow
def test_multicanonical_run_recovers_ln_omega_4x4():
    """Full method (Sec. 2) on 4x4, N=8: iterate the recursion to a flat H,
    then one long iteration; ln Omega within 0.02 of the enumeration."""
    sysm = muca.System(2, 4, 8, 32, 100)
    iters, H, f = muca.run_to_flat(sysm, 2000, 40, "recursive", t_lo=-12, t_hi=0)
    assert f >= 0.5, (iters, f)
    H, _, _ = sysm.iterate(80000, 1000)
    est = ln_omega(sysm.lnW, H, 16, 8)
    for e, c in OM.items():
        assert abs(est[e - E_LO] - math.log(c)) < 0.02, (e, est[e - E_LO], math.log(c))


def test_multicanonical_simple_scheme_flattens_3x3():
    sysm = muca.System(2, 3, 4, 16, 7)
    iters, H, f = muca.run_to_flat(sysm, 1000, 30, "simple", t_lo=-4, t_hi=-2)
    assert f >= 0.5


def test_reweighting_exact_from_exact_histogram():
    """Reweighting (Sec. 3) of an exact multicanonical histogram to any beta
    gives the canonical moments of the enumerated density of states."""
    rng = np.random.default_rng(9)
    lnW = rng.normal(size=NB)
    H = _exact_hist(OM, lnW, E_LO)
    for beta in (0.0, 0.5, 1.3, -0.4):
        e1, e2 = muca.reweight_moments(lnW, H, E_LO, beta)
        x1, x2 = muca.exact_moments(OM, beta)
        assert e1 == pytest.approx(x1, rel=1e-10)
        assert e2 == pytest.approx(x2, rel=1e-10)
    # infinite temperature: the plain average over all C(16, 8) states
    mean = sum(c * e for e, c in OM.items()) / math.comb(16, 8)
    assert muca.exact_moments(OM, 0.0)[0] == pytest.approx(mean, rel=1e-12)


def test_multi_histogram_joins_windows_exactly():
    """Two exact histograms of the 4x4, N = 8 lattice sampled with different
    weights, each seeing only part of the energy range (as from two windows)
    and with different total counts: the combination recovers ln Omega over
    the union, which needs the free energies f_k to be right."""
    from oracle.recursion import multi_histogram
    rng = np.random.default_rng(12)
    lnW1, lnW2 = rng.normal(size=NB), rng.normal(scale=2.0, size=NB)
    H1 = _exact_hist(OM, lnW1, E_LO, total=1e9)
    H2 = _exact_hist(OM, lnW2, E_LO, total=3e7)
    H1[: -8 - E_LO] = 0.0                      # window E >= -8
    H2[-5 - E_LO:] = 0.0                       # window E <= -6
    # outside its window a run has weight 0: lnW = -inf there
    w1, w2 = lnW1.copy(), lnW2.copy()
    w1[: -8 - E_LO] = -np.inf
    w2[-5 - E_LO:] = -np.inf
    lo, passes = multi_histogram(np.stack([H1, H2]), np.stack([w1, w2]))
    ideal = np.array([math.log(OM[E_LO + b]) if (E_LO + b) in OM else np.nan for b in range(NB)])
    mask = ~np.isnan(ideal)
    _agree_up_to_constant(lo, ideal, mask, 1e-8)
    assert np.isnan(lo[-11 - E_LO])
    # one histogram alone: ln H - lnW
    lo1, _ = multi_histogram(H1[None, :], lnW1[None, :])
    vis = H1 > 0
    ref = np.log(H1[vis]) - lnW1[vis]
    np.testing.assert_allclose(lo1[vis], ref - ref.max(), atol=1e-12)


def test_reweight_observable_is_canonical_enumeration():
    """An exact multicanonical histogram with the microcanonical mean of the
    largest droplet per energy, reweighted (Sec. 3), equals the canonical
    average of the largest droplet over all C(16, 8) configurations."""
    from itertools import combinations
    d, L, N, V = 2, 4, 8, 16
    per_e = {}
    configs = []
    for combo in combinations(range(V), N):
        occ = np.zeros(V, np.uint8)
        occ[list(combo)] = 1
        e = chain.energy(d, L, occ)
        vd = chain.largest_droplet(d, L, occ)
        configs.append((e, vd))
        per_e.setdefault(e, []).append(vd)
    rng = np.random.default_rng(6)
    lnW = rng.normal(size=NB)
    H = _exact_hist(OM, lnW, E_LO)
    obs = np.full(NB, np.nan)
    for e, v in per_e.items():
        obs[e - E_LO] = sum(v) / len(v)
    for beta in (0.0, 1.0, 2.5):
        w = np.array([math.exp(-beta * e) for e, _ in configs])
        ref = float((w * np.array([v for _, v in configs])).sum() / w.sum())
        assert muca.reweight_observable(lnW, H, E_LO, beta, obs) == pytest.approx(ref, rel=1e-10)


# ------------------------------------------------ edge continuation (flag) --

def test_edge_continuation_extends_canonical_weights_exactly():
    """Canonical weights lnW = -beta E on the visited members (with gaps and
    arbitrary values between members) continue as the same line beyond both
    ends: the continuation is the canonical weight at the edge's slope."""
    from oracle.recursion import extrapolate_edges
    rng = np.random.default_rng(3)
    for _ in range(20):
        nb = int(rng.integers(20, 200))
        beta = float(rng.normal(scale=2.0))
        s_cum = np.zeros(nb, bool)
        lo = int(rng.integers(1, nb // 3))
        hi = int(rng.integers(2 * nb // 3, nb - 1))
        s_cum[lo:hi + 1] = rng.random(hi - lo + 1) < 0.8
        s_cum[lo] = s_cum[hi] = True
        E = np.arange(nb) - nb
        lnW = np.where(s_cum, -beta * E, rng.normal(size=nb))
        out = extrapolate_edges(lnW, s_cum)
        shift = out[lo] - lnW[lo]
        np.testing.assert_allclose(out[:lo] - shift, -beta * E[:lo], rtol=0, atol=1e-9)
        np.testing.assert_allclose(out[hi + 1:] - shift, -beta * E[hi + 1:], rtol=0, atol=1e-9)
        # members and interior gaps keep their values (up to the common shift)
        np.testing.assert_allclose(out[lo:hi + 1] - shift, lnW[lo:hi + 1], rtol=0, atol=1e-9)
        assert out.max() == 0.0


def test_edge_continuation_by_hand():
    """Members 2..5 and 9 of 12 bins with k = 8 > members: the slopes come
    from the far ends of the member set (bins 2 and 9)."""
    from oracle.recursion import extrapolate_edges
    lnW = np.zeros(12)
    s_cum = np.zeros(12, bool)
    s_cum[[2, 3, 4, 5, 9]] = True
    lnW[[2, 3, 4, 5, 9]] = [7.0, 5.0, 4.0, 3.0, 0.0]
    out = extrapolate_edges(lnW, s_cum)
    # below: slope (lnW[9] - lnW[2]) / 7 = -1 -> bins 0, 1 take 9, 8
    # above: slope (lnW[9] - lnW[2]) / 7 = -1 -> bins 10, 11 take -1, -2
    expect = np.array([9, 8, 7, 5, 4, 3, 0, 0, 0, 0, -1, -2], dtype=float) - 9.0
    np.testing.assert_allclose(out, expect, atol=1e-12)
    # with k = 1 the slopes come from the neighbouring members
    out1 = extrapolate_edges(lnW, s_cum, k=1)
    expect1 = np.array([11, 9, 7, 5, 4, 3, 0, 0, 0, 0, -0.75, -1.5]) - 11.0
    np.testing.assert_allclose(out1, expect1, atol=1e-12)


def test_edge_continuation_needs_two_members():
    from oracle.recursion import extrapolate_edges
    lnW = np.array([3.0, 1.0, 2.0])
    s = np.array([False, True, False])
    np.testing.assert_array_equal(extrapolate_edges(lnW, s), lnW - 3.0)


@pytest.mark.slow
def test_multicanonical_run_with_edge_continuation_recovers_ln_omega_4x4():
    """The full method with the simple iteration and the edge continuation
    (from lnW = 0, 4x4, N = 8): flat, then ln Omega within 0.02 of the
    enumeration on every bin."""
    sysm = muca.System(2, 4, 8, 32, 300)
    iters, H, f = muca.run_to_flat(sysm, 2000, 40, "simple", t_lo=-12, t_hi=0, extrapolate=True)
    assert f >= 0.5, (iters, f)
    H, _, _ = sysm.iterate(80000, 1000)
    est = ln_omega(sysm.lnW, H, 16, 8)
    for e, c in OM.items():
        assert abs(est[e - E_LO] - math.log(c)) < 0.02, (e, est[e - E_LO], math.log(c))
