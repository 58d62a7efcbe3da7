"""GPU parity of the largest-droplet measurement and of the reweighting of
the library's own histograms (Sec. 3).

The walkers' configurations on both sides come from their own chains (the
oracle's walker chain is bit-exact with the device's, see the parity
tests); the oracle's breadth-first search then gives V_D per walker, and the
per-energy accumulators follow from those and the oracle's energies.  All of
it is integer work: bit-exact.
"""
import numpy as np
import pytest

from oracle import chain, muca
from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


def _weights(kind, nb):
    if kind == "random":
        return workloads.random_log_weights(nb, 1, scale=0.5)
    # favour bonds strongly: walkers condense into droplets
    return -1.2 * np.arange(nb, dtype=np.float64)


def _run_both(desc, kind, rounds, sweeps):
    """Run `rounds` iterations of `sweeps` sweeps with a measurement after
    each, on the device and in the oracle; returns (device V_D per round,
    oracle V_D per round, device accumulators, oracle accumulators)."""
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = (-d * N, 0) if lo == 0 and hi == 0 else (lo, hi)
    nb = e_hi - e_lo + 1
    lnW = _weights(kind, nb)
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    acc = np.zeros((3, nb), np.int64)
    got, want = [], []
    with m.Mucal([desc]) as mc:
        mc.set_weights(0, lnW)
        for it in range(rounds):
            mc.run_iteration(sweeps, it)
            mc.measure_droplets()
            got.append(mc.largest_droplets(0))
            chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            vd = np.array([chain.largest_droplet(d, L, occ[w]) for w in range(W)], np.int64)
            want.append(vd)
            for w in range(W):
                b = int(E[w]) - e_lo
                acc[0, b] += 1
                acc[1, b] += vd[w]
                acc[2, b] += vd[w] * vd[w]
        dev = mc.droplet_stats(0)
    return got, want, dev, acc


@pytest.mark.parametrize("desc,kind,rounds,sweeps", [
    ((2, 8, 20, 64, 0, 0, 3), "random", 3, 5),
    ((3, 5, 30, 37, 0, 0, 11), "random", 3, 5),           # ragged walker count
    ((2, 16, 40, 64, 0, 0, 5), "condense", 4, 40),        # deep union-find trees
    ((3, 8, 120, 32, 0, 0, 8), "condense", 3, 30),
    ((3, 5, 124, 4, 0, 0, 9), "random", 2, 3),            # N = V - 1: one droplet of N
    ((2, 3, 1, 5, 0, 0, 77), "random", 2, 3),             # N = 1
    ((2, 257, 2000, 4, 0, 0, 5), "random", 1, 1),         # uint32 lists, global parent array
    ((3, 40, 3000, 6, 0, 0, 21), "condense", 1, 2),       # 4 V bytes above shared memory
])
def test_largest_droplet_bit_exact(desc, kind, rounds, sweeps):
    got, want, dev, acc = _run_both(desc, kind, rounds, sweeps)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
    for k in range(3):
        np.testing.assert_array_equal(dev[k], acc[k])
    if desc[2] == desc[1] ** desc[0] - 1:
        assert (got[-1] == desc[2]).all()
    if kind == "condense" and desc[1] <= 16:
        assert max(g.max() for g in got) >= desc[2] // 2   # droplets really formed


@pytest.mark.parametrize("wl,sweeps", [(workloads.MEDIUM_2D, 20), (workloads.LARGE_3D, 2)])
def test_droplet_full_size(wl, sweeps):
    """The 64x64 (N = 410, 4096 walkers) and 32^3 (N = 3277, 8192 walkers)
    systems at weights that favour bonds: every walker's V_D and the
    accumulators against the oracle."""
    got, want, dev, acc = _run_both(wl.systems[0], "condense", 1, sweeps)
    np.testing.assert_array_equal(got[0], want[0])
    for k in range(3):
        np.testing.assert_array_equal(dev[k], acc[k])


def test_droplets_batched_systems_and_reset():
    descs = [(2, 8, 20, 16, 0, 0, 0), (3, 6, 40, 9, 0, 0, 100)]
    with m.Mucal(descs) as mc:
        with pytest.raises(m.MucalError) as e:
            mc.droplet_stats(0)
        assert e.value.code == m.MUCAL_ERR_NOT_READY
        mc.run_iteration(3, 0)
        mc.measure_droplets()
        mc.measure_droplets()
        for s, (d, L, N, W, lo, hi, seed) in enumerate(descs):
            S, occ, E = chain.init_walkers(d, L, N, W, seed)
            T = chain.thresholds(d, -d * N, 0, np.zeros(d * N + 1))
            chain.run_walkers(d, L, N, seed, 0, 3 * N, -d * N, 0, T, S, occ, E)
            vd = np.array([chain.largest_droplet(d, L, occ[w]) for w in range(W)])
            np.testing.assert_array_equal(mc.largest_droplets(s), vd)
            cnt, sm, sm2 = mc.droplet_stats(s)
            assert cnt.sum() == 2 * W and sm.sum() == 2 * vd.sum() and sm2.sum() == 2 * (vd ** 2).sum()
        mc.reset_droplet_stats()
        for s in range(2):
            assert all((a == 0).all() for a in mc.droplet_stats(s))


def test_reweight_system_uses_the_sampling_weights():
    desc = (2, 8, 20, 64, 0, 0, 3)
    nb = 41
    lnW = workloads.random_log_weights(nb, 2, scale=0.3)
    betas = [0.0, 0.7, 2.0]
    with m.Mucal([desc]) as mc:
        mc.set_weights(0, lnW)
        mc.run_iteration(10, 0)
        H = mc.histogram(0)
        a = mc.reweight(0, betas)
        mc.update_weights(0)                  # new weights; the histogram's stay
        b = mc.reweight(0, betas)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
        for i, bt in enumerate(betas):
            e1, e2 = muca.reweight_moments(lnW, H, -40, bt)
            assert a[0][i] == pytest.approx(e1, rel=1e-12)
            assert a[1][i] == pytest.approx(e2, rel=1e-12)


def test_converged_run_reweights_to_exact_canonical_moments():
    """4x4, N = 8: iterate to a flat histogram on the device, one long
    production iteration, reweight to several beta and compare <E> and the
    energy variance with the enumeration (Eq. 1)."""
    omega = chain.enumerate_omega(2, 4, 8)
    with m.Mucal([(2, 4, 8, 512, 0, 0, 7)]) as mc:
        mc.set_target_window(0, -12, 0)
        f = -1.0
        for it in range(60):
            mc.run_iteration(200, it)
            _, f = mc.update_weights(0)
            if f >= 0.5:
                break
        assert f >= 0.5
        mc.run_iteration(4000, 1000)
        betas = [0.0, 0.5, 1.0, 2.0]
        mE, mE2 = mc.reweight(0, betas)
    for i, bt in enumerate(betas):
        x1, x2 = muca.exact_moments(omega, bt)
        assert mE[i] == pytest.approx(x1, abs=0.03), bt
        var, xvar = mE2[i] - mE[i] ** 2, x2 - x1 ** 2
        assert var == pytest.approx(xvar, rel=0.03), bt


def test_multi_histogram_ln_omega_from_iterations():
    """4x4, N = 8: ln Omega combined from the last 12 of 20 iterations of the
    weight recursion (multi-histogram, each histogram with the weights it was
    sampled with) within 0.02 of the enumeration on every bin."""
    import math
    from paper_1401_4076_gb300 import iterate
    omega = chain.enumerate_omega(2, 4, 8)
    res = iterate.iterate_to_flat([(2, 4, 8, 512, 0, 0, 31)], sweeps=400, max_iter=20,
                                  targets=[(-12, 0)], goal=2.0, history=12)[0]
    assert len(res.extra["history"]) == 12
    lo = iterate.ln_omega_multi(res.extra["history"], 16, 8)
    for e, c in omega.items():
        assert abs(lo[e + 16] - math.log(c)) < 0.02, (e, lo[e + 16], math.log(c))


def test_production_curve_against_enumeration():
    """4x4, N = 8: flat weights, production with droplet measurements, then
    <E>, the specific heat and <V_D> reweighted to a grid of temperatures,
    against the canonical sums over all C(16, 8) configurations."""
    import math
    from itertools import combinations
    from paper_1401_4076_gb300 import production
    d, L, N, V = 2, 4, 8, 16
    temps = [0.4, 0.7, 1.0, 2.0]
    res = production.run((d, L, N, 512, 0, 0, 17), temps, sweeps=400, max_iter=100,
                         prod_rounds=20, prod_sweeps=1000, target=(-12, 0))
    assert res["converged"]
    cfg = []
    for combo in combinations(range(V), N):
        occ = np.zeros(V, np.uint8)
        occ[list(combo)] = 1
        cfg.append((chain.energy(d, L, occ), chain.largest_droplet(d, L, occ)))
    E = np.array([e for e, _ in cfg], float)
    D = np.array([v for _, v in cfg], float)
    for row in res["curve"]:
        w = np.exp(-(E - E.min()) / row["T"])
        e1 = (w * E).sum() / w.sum()
        e2 = (w * E * E).sum() / w.sum()
        cv = (e2 - e1 * e1) / (row["T"] ** 2 * V)
        assert row["mean_E"] == pytest.approx(e1, abs=0.03), row
        assert row["specific_heat_per_site"] == pytest.approx(cv, rel=0.05, abs=2e-3), row
        assert row["mean_V_D"] == pytest.approx((w * D).sum() / w.sum(), abs=0.05), row
        assert row["mean_E_ising"] == pytest.approx(4 * (row["mean_E"] - muca.ising_constant(d, L, N)))
