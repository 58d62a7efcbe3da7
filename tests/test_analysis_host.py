"""Host-side analysis functions of libmucal against the oracle (no GPU).

mucal_reweight, mucal_droplet_delta and mucal_droplet_lambda run in double
precision on the host; they are compared with the oracle's plain versions
(Sec. 3, Eqs. 1 and 8-10) and with brute-force sums over every configuration
of a small lattice.
"""
import math
import os
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest

from oracle import chain, droplet, muca
from paper_1401_4076_gb300 import mucal as m

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    return m.load_library()


def test_reweight_matches_oracle_on_random_histograms():
    rng = np.random.default_rng(5)
    for nb in (1, 7, 41, 300):
        H = rng.integers(0, 10 ** 9, nb)
        H[rng.random(nb) < 0.3] = 0
        H[rng.integers(nb)] = 17
        lnW = rng.normal(scale=30.0, size=nb)
        e_lo = -int(rng.integers(0, 2 * nb))
        betas = np.array([0.0, 0.3, 2.6667, -1.0, 7.0])
        obs = rng.normal(size=(2, nb))
        obs[1, rng.random(nb) < 0.4] = np.nan
        mE, mE2, out = m.mucal_reweight(H, lnW, e_lo, betas, obs)
        for i, bt in enumerate(betas):
            e1, e2 = muca.reweight_moments(lnW, H, e_lo, bt)
            assert mE[i] == pytest.approx(e1, rel=1e-12, abs=1e-12)
            assert mE2[i] == pytest.approx(e2, rel=1e-12, abs=1e-12)
            for k in range(2):
                ref = muca.reweight_observable(lnW, H, e_lo, bt, obs[k])
                if math.isnan(ref):
                    assert math.isnan(out[i, k])
                else:
                    assert out[i, k] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_reweight_of_exact_histogram_is_canonical_enumeration():
    """4x4, N = 8: an exact multicanonical histogram with arbitrary weights,
    reweighted, gives <E>, <E^2> and <V_D> equal to the plain canonical sums
    over all C(16, 8) configurations."""
    d, L, N, V = 2, 4, 8, 16
    e_lo = -d * N
    nb = d * N + 1
    per_e = {}
    configs = []
    for combo in combinations(range(V), N):
        occ = np.zeros(V, np.uint8)
        occ[list(combo)] = 1
        e = chain.energy(d, L, occ)
        vd = chain.largest_droplet(d, L, occ)
        configs.append((e, vd))
        per_e.setdefault(e, []).append(vd)
    rng = np.random.default_rng(3)
    lnW = rng.normal(size=nb)
    H = np.zeros(nb, np.int64)
    obs = np.full(nb, np.nan)
    scale = 1e12
    z0 = sum(len(v) * math.exp(lnW[e - e_lo]) for e, v in per_e.items())
    for e, v in per_e.items():
        H[e - e_lo] = int(round(scale * len(v) * math.exp(lnW[e - e_lo]) / z0))
        obs[e - e_lo] = sum(v) / len(v)
    for beta in (0.0, 0.8, 2.0):
        mE, mE2, out = m.mucal_reweight(H, lnW, e_lo, [beta], obs[None, :])
        w = np.array([math.exp(-beta * e) for e, _ in configs])
        E = np.array([e for e, _ in configs], float)
        D = np.array([v for _, v in configs], float)
        # H is rounded to integers of order 1e12, so agreement is to ~1e-10
        assert mE[0] == pytest.approx((w * E).sum() / w.sum(), rel=1e-9)
        assert mE2[0] == pytest.approx((w * E * E).sum() / w.sum(), rel=1e-9)
        assert out[0, 0] == pytest.approx((w * D).sum() / w.sum(), rel=1e-9)


def test_reweight_rejects_bad_input():
    H = np.array([0, 3, 4])
    w = np.zeros(3)
    with pytest.raises(m.MucalError):
        m.mucal_reweight(np.zeros(3, np.int64), w, 0, [1.0])
    with pytest.raises(m.MucalError):
        m.mucal_reweight(np.array([1, -1, 2]), w, 0, [1.0])
    with pytest.raises(m.MucalError):
        m.mucal_reweight(H, np.array([0.0, np.inf, 0.0]), 0, [1.0])
    with pytest.raises(m.MucalError):
        m.mucal_reweight(H, w, 0, [np.nan])
    assert "beta" in m.mucal_last_error(None)


def test_droplet_delta_matches_oracle():
    for d, V, N, rho0, kap, tau in ((2, 6400, 100, 0.00675, 0.02708, 1.06125),
                                    (3, 32768, 300, 0.002739, 0.00608, 2.861),
                                    (2, 100, 0, 0.0, 1.0, 1.0), (3, 1000, 2, 0.01, 0.1, 0.2)):
        D, vl = m.mucal_droplet_delta(d, V, N, rho0, kap, tau)
        assert vl == pytest.approx(droplet.excess_volume(V, N, rho0), rel=1e-14, abs=1e-14)
        assert D == pytest.approx(droplet.delta(d, V, N, rho0, kap, tau), rel=1e-13, abs=0)
    with pytest.raises(m.MucalError):
        m.mucal_droplet_delta(4, 10, 1, 0.0, 1.0, 1.0)
    with pytest.raises(m.MucalError):
        m.mucal_droplet_delta(2, 10, 1, 0.5, 1.0, 1.0)


def test_droplet_lambda_matches_brute_force():
    for d in (2, 3):
        dc = (1 / d) * ((d + 1) / 2) ** ((d + 1) / d)
        for D in np.concatenate([np.linspace(0, 3, 61), [5.0, 10.0, 50.0, 1e3]]):
            if abs(D - dc) < 1e-3:
                continue
            ref = droplet.lambda_of_delta(d, D)
            assert m.mucal_droplet_lambda(d, D) == pytest.approx(ref, abs=1e-6), (d, D)
    with pytest.raises(m.MucalError):
        m.mucal_droplet_lambda(2, -1.0)


def test_droplet_lambda_critical_point_is_the_printed_one():
    """The library's jump location, found by bisection on its output, against
    the Delta_c and lambda_c printed in Sec. 3."""
    for line in open(os.path.join(GOLDEN, "droplet_critical.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        d, dc, lc = line.split()
        d, dc, lc = int(d), float(dc), float(Fraction(lc))
        lo, hi = 0.5, 1.5
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if m.mucal_droplet_lambda(d, mid) > 0:
                hi = mid
            else:
                lo = mid
        assert hi == pytest.approx(dc, abs=5e-5)
        assert m.mucal_droplet_lambda(d, hi) == pytest.approx(lc, abs=1e-6)


def test_table1_constants_as_printed():
    """The condensation pipeline's Table 1 constants against the printed
    table (tests/golden/table1_parameters.txt)."""
    from paper_1401_4076_gb300 import condensation
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_parameters.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for d, T, rho0, kap, tau in rows:
        t = condensation.TABLE1[int(d)]
        assert (t["T"], t["rho0"], t["kappa_hat"], t["tau_W"]) == (float(T), float(rho0), float(kap),
                                                                    float(tau))


def test_multi_histogram_matches_oracle():
    from oracle.recursion import multi_histogram
    rng = np.random.default_rng(21)
    for K, nb in ((1, 30), (3, 60), (4, 90)):
        H = rng.integers(0, 10 ** 6, (K, nb))
        lnW = rng.normal(scale=5.0, size=(K, nb))
        for k in range(K):                     # each run sees a window of its own
            lo = int(rng.integers(0, nb // 2))
            hi = int(rng.integers(nb // 2, nb))
            H[k, :lo] = 0
            H[k, hi:] = 0
            lnW[k, :lo] = -np.inf
            lnW[k, hi:] = -np.inf
        H[:, 7] = 0                            # a bin no run visits
        got, passes = m.mucal_multi_histogram(H, lnW, max_iter=5000, tol=1e-13)
        ref, ref_passes = multi_histogram(H, lnW, max_iter=5000, tol=1e-13)
        assert np.isnan(got[7]) and np.isnan(ref[7])
        ok = ~np.isnan(ref)
        np.testing.assert_allclose(got[ok], ref[ok], rtol=0, atol=1e-9)
        assert passes == ref_passes
    with pytest.raises(m.MucalError):
        m.mucal_multi_histogram(np.zeros((2, 5), np.int64), np.zeros((2, 5)))


def test_ising_constant_matches_oracle():
    for d, L, N in ((2, 4, 8), (3, 5, 40), (2, 64, 410)):
        V = L ** d
        assert m.mucal_ising_constant(d, V, N) == pytest.approx(muca.ising_constant(d, L, N), rel=1e-15)
    with pytest.raises(m.MucalError):
        m.mucal_ising_constant(4, 10, 1)


# ------------------------------------- context-free weight update and ln Omega

def _histogram_sequence(nb, n_iter, seed):
    """Histograms whose visited range grows and moves, with gaps and zeros."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_iter):
        H = np.zeros(nb, dtype=np.int64)
        lo = max(0, nb // 2 - 3 * i - int(rng.integers(0, 3)))
        hi = min(nb, nb // 2 + 2 * i + 5)
        H[lo:hi] = rng.integers(1, 10 ** 7, hi - lo)
        H[lo + rng.integers(0, max(1, hi - lo), 2)] = 0
        out.append(H)
    return out


@pytest.mark.parametrize("nb", [1, 9, 161])
def test_weight_update_matches_oracle_recursion(nb):
    """mucal_weight_update (the code the contexts run) against the oracle's
    recursion and simple iteration of Sec. 2: weights to 1e-12, visited set
    and accumulated pair weights, flatness."""
    from oracle.recursion import flatness, recursive_update, simple_update
    seq = _histogram_sequence(nb, 12, nb)
    st = m.WeightState(nb)
    lnW = np.zeros(nb)
    s_cum = np.zeros(nb, bool)
    phat = np.zeros(nb)
    for H in seq:
        f = m.mucal_weight_update(st, H, m.MUCAL_SCHEME_RECURSIVE)
        lnW, s_cum, phat = recursive_update(lnW, H, s_cum, phat)
        np.testing.assert_allclose(st.lnW, lnW, rtol=1e-12, atol=1e-12 * max(1, np.abs(lnW).max()))
        np.testing.assert_array_equal(st.visited.astype(bool), s_cum)
        np.testing.assert_allclose(st.pacc, phat, rtol=1e-12)
        assert f == pytest.approx(flatness(H, s_cum), rel=1e-15, abs=0)
    st = m.WeightState(nb)
    lnW = np.zeros(nb)
    for H in seq:
        m.mucal_weight_update(st, H, m.MUCAL_SCHEME_SIMPLE)
        lnW = simple_update(lnW, H)
        np.testing.assert_allclose(st.lnW, lnW, rtol=1e-12, atol=1e-12 * max(1, np.abs(lnW).max()))


def test_weight_update_target_window_and_errors():
    from oracle.recursion import flatness
    H = np.array([0, 5, 10, 20, 0, 40], dtype=np.int64)
    st = m.WeightState(6)
    f = m.mucal_weight_update(st, H, m.MUCAL_SCHEME_RECURSIVE, target=(1, 3))
    assert f == pytest.approx(flatness(H, st.visited.astype(bool), 1, 3)) == 0.25
    st2 = m.WeightState(6)
    assert m.mucal_weight_update(st2, H, m.MUCAL_SCHEME_RECURSIVE, target=(0, 3)) == -1.0
    with pytest.raises(m.MucalError):
        m.mucal_weight_update(m.WeightState(6), H, 7)
    with pytest.raises(m.MucalError):
        m.mucal_weight_update(m.WeightState(6), -H, m.MUCAL_SCHEME_SIMPLE)
    with pytest.raises(m.MucalError):
        m.mucal_weight_update(m.WeightState(6), H, m.MUCAL_SCHEME_SIMPLE, target=(2, 9))


def test_ln_omega_matches_oracle():
    """O8: ln Omega = ln H - lnW on visited bins, normalised to C(V, N)."""
    from oracle.recursion import ln_omega
    rng = np.random.default_rng(11)
    for V, N, nb in ((16, 8, 13), (4096, 410, 821), (110592, 11059, 300)):
        H = rng.integers(0, 10 ** 9, nb)
        H[rng.random(nb) < 0.2] = 0
        H[0] = 3
        lnW = rng.normal(scale=50.0, size=nb)
        got = m.mucal_ln_omega(H, lnW, V, N)
        ref = ln_omega(lnW, H, V, N)
        np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
        v = ~np.isnan(ref)
        np.testing.assert_allclose(got[v], ref[v], rtol=1e-12, atol=1e-12 * np.abs(ref[v]).max())
    with pytest.raises(m.MucalError):
        m.mucal_ln_omega(np.zeros(4, np.int64), np.zeros(4), 16, 8)


def test_ln_omega_of_exact_enumeration():
    """With the exact multicanonical histogram H = Omega W (4x4, N = 8), the
    estimate returns the enumerated ln Omega itself."""
    om = chain.enumerate_omega(2, 4, 8)
    nb = 2 * 8 + 1
    Om = np.zeros(nb)
    for e, c in om.items():
        Om[e + 16] = c
    lnW = np.where(Om > 0, -np.log(np.where(Om > 0, Om, 1)), 0.0)
    H = np.where(Om > 0, 1000, 0).astype(np.int64)       # flat: H = Omega W x 1000
    got = m.mucal_ln_omega(H, lnW, 16, 8)
    v = Om > 0
    np.testing.assert_allclose(got[v], np.log(Om[v]), rtol=0, atol=1e-12)
    assert np.isnan(got[~v]).all()


def test_ln_omega_normalise_of_multi_histogram_matches_oracle():
    from oracle.recursion import multi_histogram
    rng = np.random.default_rng(3)
    nb = 60
    H = rng.integers(1, 10 ** 6, (3, nb))
    H[0, :10] = 0
    W = rng.normal(scale=5.0, size=(3, nb))
    lo, _ = m.mucal_multi_histogram(H, W)
    ref, _ = multi_histogram(H, W)
    got = m.mucal_ln_omega_normalise(lo, 1000, 100)
    # the oracle's combination normalised by its own definition: logsumexp = ln C(V, N)
    v = ~np.isnan(ref)
    shift = (math.lgamma(1001) - math.lgamma(101) - math.lgamma(901)) - np.logaddexp.reduce(ref[v])
    np.testing.assert_allclose(got[v], ref[v] + shift, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("base", ["simple", "recursive"])
def test_weight_update_with_edge_continuation_matches_oracle(base):
    """MUCAL_SCHEME_EXTRAPOLATE or-ed with either scheme against the oracle's
    update followed by its edge continuation, over a sequence whose visited
    range grows at both ends."""
    from oracle.recursion import extrapolate_edges, recursive_update, simple_update
    nb = 201
    seq = _histogram_sequence(nb, 15, 77)
    scheme = (m.MUCAL_SCHEME_SIMPLE if base == "simple" else m.MUCAL_SCHEME_RECURSIVE)
    st = m.WeightState(nb)
    lnW = np.zeros(nb)
    s_cum = np.zeros(nb, bool)
    phat = np.zeros(nb)
    for H in seq:
        m.mucal_weight_update(st, H, scheme | m.MUCAL_SCHEME_EXTRAPOLATE)
        if base == "simple":
            s_cum = s_cum | (H > 0)
            lnW = simple_update(lnW, H)
        else:
            lnW, s_cum, phat = recursive_update(lnW, H, s_cum, phat)
        lnW = extrapolate_edges(lnW, s_cum)
        np.testing.assert_allclose(st.lnW, lnW, rtol=1e-12, atol=1e-12 * max(1, np.abs(lnW).max()))
    with pytest.raises(m.MucalError):
        m.mucal_weight_update(m.WeightState(nb), seq[0], 0x20)
