"""GPU parity: the CUDA path through the C ABI against the oracle.

Integer work (placement, thresholds, walker chains, histograms) must be
bit-exact; the float64 weight iteration must agree to 1e-12 relative.  Small
systems are compared in full (every walker, every iteration); the large
workloads in the launch configuration the benchmark times are compared on
sampled walkers, whose final states and histograms the oracle computes one by
one, and through invariants that hold at any size.
"""
import numpy as np
import pytest

from oracle import chain
from oracle.recursion import recursive_update, simple_update
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


def _window(d, N, e_lo, e_hi):
    return (-d * N, 0) if (e_lo == 0 and e_hi == 0) else (e_lo, e_hi)


def _oracle_states(d, L, N, walkers, seed_base, pick=None):
    S, occ, E = chain.init_walkers(d, L, N, walkers, seed_base)
    if pick is not None:
        S, occ, E = S[pick].copy(), occ[pick].copy(), E[pick].copy()
    return S, occ, E


def _assert_walker_equal(mc, sys, w, S, occ, E):
    g_occ, g_S, g_E = mc.walker_state(sys, w)
    np.testing.assert_array_equal(g_occ, occ)
    np.testing.assert_array_equal(g_S, S)
    assert g_E == E


def _rel_close(a, b, rtol=1e-12):
    scale = max(1.0, float(np.abs(b).max()))
    np.testing.assert_allclose(a, b, rtol=rtol, atol=rtol * scale)


# --------------------------------------------------------------- placement --

@pytest.mark.parametrize("desc", [
    (2, 16, 32, 64, 0, 0, 0),       # small 2D, uint16 lists
    (3, 8, 50, 37, 0, 0, 1000),     # ragged walker count
    (2, 257, 300, 3, 0, 0, 5),      # V = 66049 > 65536: uint32 lists
    (3, 5, 124, 4, 0, 0, 9),        # N = V - 1
    (2, 3, 1, 5, 0, 0, 77),         # L = 3, N = 1
])
def test_initial_placement_bit_exact(desc):
    d, L, N, W, lo, hi, seed = desc
    with m.Mucal([desc]) as mc:
        S, occ, E = _oracle_states(d, L, N, W, seed)
        for w in range(W):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])


# -------------------------------------------------------------- thresholds --

@pytest.mark.parametrize("d,N", [(2, 32), (3, 100)])
def test_threshold_table_bit_exact(d, N):
    L = 16 if d == 2 else 10
    with m.Mucal([(d, L, N, 2, 0, 0, 0)]) as mc:
        nb = d * N + 1
        for seed in range(3):
            lnW = workloads.random_log_weights(nb, seed, scale=0.4)
            mc.set_weights(0, lnW)
            np.testing.assert_array_equal(mc.thresholds(0), chain.thresholds(d, -d * N, 0, lnW))


# ------------------------------------------------- full small-case parity --

LAUNCHES = [
    dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=32, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=7, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=2, walkers_per_block=16, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4, walkers_per_block=24, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=32, walkers_per_block=5, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=2, walkers_per_block=16, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=4, walkers_per_block=24, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=32, walkers_per_block=1, bits_in_smem=1),
]
GROUP8 = LAUNCHES[4]
GROUP32 = LAUNCHES[6]
FIELD8 = LAUNCHES[7]
FIELD4 = LAUNCHES[9]
FIELD32 = LAUNCHES[11]


def _lid(c):
    return f"k{c['kernel']}-G{c['lanes_per_walker']}-w{c['walkers_per_block']}-s{c['bits_in_smem']}"


@pytest.mark.parametrize("launch", LAUNCHES, ids=_lid)
def test_small_2d_ten_iterations_bit_exact(launch):
    """2D L=16, N=32, 64 walkers, seeds 0..63, lnW=0 start, 10 iterations of
    2000 sweeps with the recursive update: every per-walker histogram of every
    iteration bit-exact, weights within 1e-12, thresholds bit-exact."""
    wl = workloads.SMALL_2D
    d, L, N, W, lo, hi, seed = wl.systems[0]
    e_lo, e_hi = _window(d, N, lo, hi)
    nb = e_hi - e_lo + 1
    S, occ, E = _oracle_states(d, L, N, W, seed)
    lnW = np.zeros(nb)
    s_cum = np.zeros(nb, bool)
    phat = np.zeros(nb)
    with m.Mucal(wl.systems, per_walker_hist=True) as mc:
        mc.set_launch(**launch)
        for it in range(wl.iterations):
            T = chain.thresholds(d, e_lo, e_hi, lnW)
            np.testing.assert_array_equal(mc.thresholds(0), T)
            mc.run_iteration(wl.sweeps, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, wl.sweeps * N, e_lo, e_hi, T, S, occ, E)
            H, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
            np.testing.assert_array_equal(H, hist.sum(axis=0))
            g_lnW, flat = mc.update_weights(0, m.MUCAL_SCHEME_RECURSIVE)
            lnW, s_cum, phat = recursive_update(lnW, hist.sum(axis=0), s_cum, phat)
            _rel_close(g_lnW, lnW)
        for w in (0, 31, 63):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])
        st = mc.stats(0)
        assert st["attempts"] == W * wl.sweeps * N


def test_simple_scheme_matches_oracle():
    d, L, N, W = 2, 12, 20, 16
    with m.Mucal([(d, L, N, W, 0, 0, 3)]) as mc:
        nb = d * N + 1
        lnW = np.zeros(nb)
        for it in range(4):
            mc.run_iteration(50, it)
            H = mc.histogram(0)
            g, _ = mc.update_weights(0, m.MUCAL_SCHEME_SIMPLE)
            lnW = simple_update(lnW, H)
            _rel_close(g, lnW)


# ---------------------------------------------------------- edge cases ------

@pytest.mark.parametrize("launch", [LAUNCHES[0], LAUNCHES[3], GROUP32, FIELD4, FIELD32], ids=_lid)
@pytest.mark.parametrize("desc,sweeps", [
    ((3, 6, 40, 37, 0, 0, 11), 30),          # 3D, ragged walker count
    ((2, 3, 1, 5, 0, 0, 77), 200),           # single particle on 3x3
    ((3, 5, 124, 4, 0, 0, 9), 20),           # N = V - 1: one hole
    ((2, 257, 300, 2, 0, 0, 5), 3),          # uint32 site lists
    ((3, 4, 20, 8, -30, -2, 0), 40),         # user window (checked to hold the start)
    ((2, 8, 3, 9, 0, 0, 3), 7),              # attempts per walker (21) not a multiple of G
])
def test_edge_cases_bit_exact(desc, sweeps, launch):
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = _window(d, N, lo, hi)
    nb = e_hi - e_lo + 1
    S, occ, E = _oracle_states(d, L, N, W, seed)
    if lo or hi:
        if not ((E >= e_lo) & (E <= e_hi)).all():
            with pytest.raises(m.MucalError):
                m.Mucal([desc])
            return
    lnW = workloads.random_log_weights(nb, 1, scale=0.5)
    with m.Mucal([desc], per_walker_hist=True) as mc:
        try:
            mc.set_launch(**launch)
        except m.MucalError:
            if launch["kernel"] == m.MUCAL_KERNEL_FIELD:
                # the fields of a whole warp of walkers do not fit: one walker per block
                mc.set_launch(**dict(launch, lanes_per_walker=32, walkers_per_block=1))
            else:                   # bitsets too large for shared memory at this block size
                mc.set_launch(**dict(launch, bits_in_smem=0))
        mc.set_weights(0, lnW)
        T = chain.thresholds(d, e_lo, e_hi, lnW)
        for it in range(2):
            mc.run_iteration(sweeps, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            _, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
        for w in range(W):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])


def test_window_boundary_is_never_crossed():
    """A narrow window around the start: moves leaving it are rejected (T = 0)."""
    d, L, N, W, seed = 2, 10, 30, 16, 4
    S, occ, E = _oracle_states(d, L, N, W, seed)
    e_lo, e_hi = int(E.min()) - 2, int(E.max()) + 2
    e_hi = min(e_hi, 0)
    desc = (d, L, N, W, e_lo, e_hi, seed)
    T = chain.thresholds(d, e_lo, e_hi, np.zeros(e_hi - e_lo + 1))
    with m.Mucal([desc], per_walker_hist=True) as mc:
        mc.run_iteration(100, 0)
        _, per = mc.histogram(0, per_walker=True)
    hist, _ = chain.run_walkers(d, L, N, seed, 0, 100 * N, e_lo, e_hi, T, S, occ, E)
    np.testing.assert_array_equal(per, hist)
    assert per[:, 0].sum() > 0 or per[:, -1].sum() > 0


# ------------------------------------------------ several systems, one launch

@pytest.mark.parametrize("launch", [LAUNCHES[0], GROUP8, FIELD8], ids=_lid)
def test_multi_system_launch_bit_exact(launch):
    systems = [(2, 16, 32, 40, 0, 0, 0), (3, 8, 60, 25, 0, 0, 500), (2, 24, 50, 33, 0, 0, 900)]
    with m.Mucal(systems, per_walker_hist=True) as mc:
        mc.set_launch(**launch)
        lnWs = []
        for i, (d, L, N, W, lo, hi, seed) in enumerate(systems):
            lnW = workloads.random_log_weights(d * N + 1, 10 + i, scale=0.3)
            mc.set_weights(i, lnW)
            lnWs.append(lnW)
        mc.run_iteration(25, 3)
        for i, (d, L, N, W, lo, hi, seed) in enumerate(systems):
            S, occ, E = _oracle_states(d, L, N, W, seed)
            T = chain.thresholds(d, -d * N, 0, lnWs[i])
            hist, _ = chain.run_walkers(d, L, N, seed, 3, 25 * N, -d * N, 0, T, S, occ, E)
            H, per = mc.histogram(i, per_walker=True)
            np.testing.assert_array_equal(per, hist)
            np.testing.assert_array_equal(H, hist.sum(axis=0))


# -------------------------------------------- full-size, sampled walkers ----

def _sampled_full_size(wl, sweeps, pick, launch=None, lnW_seed=None):
    d, L, N, W, lo, hi, seed = wl.systems[0]
    e_lo, e_hi = _window(d, N, lo, hi)
    nb = e_hi - e_lo + 1
    lnW = np.zeros(nb) if lnW_seed is None else workloads.random_log_weights(nb, lnW_seed, 0.05)
    with m.Mucal(wl.systems, per_walker_hist=True) as mc:
        if launch:
            mc.set_launch(**launch)
        mc.set_weights(0, lnW)
        mc.run_iteration(sweeps, 0)
        H, per = mc.histogram(0, per_walker=True)
        assert H.sum() == W * sweeps * N
        np.testing.assert_array_equal(H, per.sum(axis=0))
        S, occ, E = _oracle_states(d, L, N, W, seed, pick)
        T = chain.thresholds(d, e_lo, e_hi, lnW)
        hist, _ = chain.run_walkers(d, L, N, seed, 0, sweeps * N, e_lo, e_hi, T, S, occ, E,
                                    walkers=pick)
        np.testing.assert_array_equal(per[pick], hist)
        for i, w in enumerate(pick):
            _assert_walker_equal(mc, 0, w, S[i], occ[i], E[i])


@pytest.mark.parametrize("launch", [None, GROUP8, dict(FIELD8, walkers_per_block=28)],
                         ids=["default", "G8", "field-G8"])
def test_medium_2d_first_iteration_sampled(launch):
    """2D L=64, N=410, 4096 walkers, first iteration (lnW = 0) at full size."""
    _sampled_full_size(workloads.MEDIUM_2D, workloads.MEDIUM_2D.sweeps, [0, 1, 777, 2048, 4095],
                       launch=launch)


@pytest.mark.parametrize("launch", [None, GROUP32, dict(FIELD8, walkers_per_block=4)],
                         ids=["default", "G32", "field-G8"])
def test_large_3d_first_iteration_sampled(launch):
    """3D L=32, N=3277, 8192 walkers, one iteration with non-trivial weights."""
    _sampled_full_size(workloads.LARGE_3D, 20, [0, 4097, 8191], launch=launch, lnW_seed=3)


# ------------------------------------- production mode (per-block rows) -----

def _lid_mc(c):
    return _lid(c) + ("-mc" if c.get("multi_commit") else "")


@pytest.mark.parametrize("launch", [LAUNCHES[0], LAUNCHES[3], GROUP8, GROUP32, FIELD8,
                                    dict(GROUP8, multi_commit=1), dict(FIELD8, multi_commit=1),
                                    dict(LAUNCHES[3], multi_commit=1)], ids=_lid_mc)
def test_production_histogram_equals_oracle_sum(launch):
    """Without per-walker histograms the rows are per block; H must still be the
    exact sum of every walker's histogram (Eq. 2)."""
    wl = workloads.SMALL_2D
    d, L, N, W, lo, hi, seed = wl.systems[0]
    lnW = workloads.random_log_weights(d * N + 1, 5, scale=0.2)
    S, occ, E = _oracle_states(d, L, N, W, seed)
    T = chain.thresholds(d, -d * N, 0, lnW)
    with m.Mucal(wl.systems) as mc:
        mc.set_launch(**launch)
        mc.set_weights(0, lnW)
        for it in range(2):
            mc.run_iteration(300, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, 300 * N, -d * N, 0, T, S, occ, E)
            np.testing.assert_array_equal(mc.histogram(0), hist.sum(axis=0))


@pytest.mark.parametrize("wl,sweeps,pick,launch", [
    (workloads.MEDIUM_2D, 200, [0, 1500, 4095],
     dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=16, bits_in_smem=1)),
    (workloads.LARGE_3D, 10, [0, 8191],
     dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=28, bits_in_smem=1)),
    (workloads.MEDIUM_2D, 200, [0, 1500, 4095],
     dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=28, bits_in_smem=1)),
], ids=["medium2d", "large3d", "medium2d-field"])
def test_full_size_production_sampled_states(wl, sweeps, pick, launch):
    """Full-size workloads in production mode: every walker's final state of a
    sample equals the oracle's, and sum H counts every attempt."""
    d, L, N, W, lo, hi, seed = wl.systems[0]
    nb = d * N + 1
    lnW = workloads.random_log_weights(nb, 8, 0.02)
    with m.Mucal(wl.systems) as mc:
        mc.set_launch(**launch)
        mc.set_weights(0, lnW)
        mc.run_iteration(sweeps, 4)
        H = mc.histogram(0)
        assert H.sum() == W * sweeps * N
        S, occ, E = _oracle_states(d, L, N, W, seed, pick)
        T = chain.thresholds(d, -d * N, 0, lnW)
        hist, _ = chain.run_walkers(d, L, N, seed, 4, sweeps * N, -d * N, 0, T, S, occ, E,
                                    walkers=pick)
        assert (H >= hist.sum(axis=0)).all()
        for i, w in enumerate(pick):
            _assert_walker_equal(mc, 0, w, S[i], occ[i], E[i])


@pytest.mark.parametrize("launch", [
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16, walkers_per_block=8, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1),
], ids=["group", "field"])
def test_batched_uneven_systems_full_size_sampled(launch):
    """The 27-system batch (2D L 32..128, 3D L 16..40, rho 0.02..0.1, 16384
    walkers) in one launch, in the launch shape the benchmark picks for it and
    with the field kernel: per system sum H counts every attempt and sampled
    walkers of every system end in the oracle's state."""
    wl = workloads.batched_uneven()
    sweeps = 5
    with m.Mucal(wl.systems) as mc:
        mc.set_launch(**launch)
        lnWs = []
        for i, (d, L, N, W, lo, hi, seed) in enumerate(wl.systems):
            lnW = workloads.random_log_weights(d * N + 1, 100 + i, scale=0.05)
            mc.set_weights(i, lnW)
            lnWs.append(lnW)
        mc.run_iteration(sweeps, 9)
        for i, (d, L, N, W, lo, hi, seed) in enumerate(wl.systems):
            H = mc.histogram(i)
            assert H.sum() == W * sweeps * N
            pick = sorted({0, W // 2, W - 1})
            S, occ, E = _oracle_states(d, L, N, W, seed, pick)
            T = chain.thresholds(d, -d * N, 0, lnWs[i])
            hist, _ = chain.run_walkers(d, L, N, seed, 9, sweeps * N, -d * N, 0, T, S, occ, E,
                                        walkers=pick)
            assert (H >= hist.sum(axis=0)).all()
            for q, w in enumerate(pick):
                _assert_walker_equal(mc, i, w, S[q], occ[q], E[q])


# ------------------------ full size, every walker, in the benchmark shapes --
# The launch shapes the benchmark's autotuner picks on GB300 (kernel, lanes
# per walker, walkers per block, bitsets in shared memory, persistent), plus
# whatever the autotuner picks live for the same weights.

BENCH_SHAPES = {
    "2d-L64-N410-w4096": dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8,
                              walkers_per_block=28, bits_in_smem=1, persistent=0),
    "3d-L32-N3277-w8192": dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4,
                               walkers_per_block=56, bits_in_smem=1, persistent=1),
    "batched-27-systems-w16384": dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16,
                                      walkers_per_block=8, bits_in_smem=1, persistent=0),
}


def _tuned_shape(systems, lnWs):
    from paper_1401_4076_gb300.autotune import autotune
    best, _ = autotune(systems, lnW=lnWs, sweeps=5, repeats=2, finalists=3)
    return best


def _every_walker_one_iteration(systems, sys_ids, sweeps, it, launch, lnWs):
    """One iteration of every system in one launch; for the systems in
    sys_ids every walker's histogram and final state against the oracle."""
    with m.Mucal(systems, per_walker_hist=True) as mc:
        mc.set_launch(**launch)
        for i, lnW in enumerate(lnWs):
            mc.set_weights(i, lnW)
        mc.run_iteration(sweeps, it)
        for i in sys_ids:
            d, L, N, W, lo, hi, seed = systems[i]
            e_lo, e_hi = _window(d, N, lo, hi)
            H, per = mc.histogram(i, per_walker=True)
            assert H.sum() == W * sweeps * N
            S, occ, E = _oracle_states(d, L, N, W, seed)
            T = chain.thresholds(d, e_lo, e_hi, lnWs[i])
            np.testing.assert_array_equal(mc.thresholds(i), T)
            hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            np.testing.assert_array_equal(per, hist)
            np.testing.assert_array_equal(H, hist.sum(axis=0))
            for w in range(W):
                _assert_walker_equal(mc, i, w, S[w], occ[w], E[w])


@pytest.mark.parametrize("shape", ["bench", "tuned"])
def test_medium_2d_every_walker_first_iteration(shape):
    """2D L=64, N=410, 4096 walkers, the first iteration from lnW = 0 at the
    benchmark's 1000 sweeps (410 000 attempts per walker): all 4096
    per-walker histograms and final states bit-exact (Eq. 2 summed on the
    device equals the oracle's sum)."""
    wl = workloads.MEDIUM_2D
    d, L, N, W, lo, hi, seed = wl.systems[0]
    lnWs = [np.zeros(d * N + 1)]
    launch = BENCH_SHAPES[wl.name] if shape == "bench" else _tuned_shape(wl.systems, lnWs)
    _every_walker_one_iteration(wl.systems, [0], wl.sweeps, 0, launch, lnWs)


@pytest.mark.parametrize("shape", ["bench", "tuned"])
def test_large_3d_every_walker_of_a_block_range(shape):
    """3D L=32, N=3277, 8192 walkers in one launch with non-trivial weights:
    256 walkers spread over the launch (every 32nd, so every block of the
    shape holds some) compared with the oracle one by one, sum H counts every
    attempt."""
    wl = workloads.LARGE_3D
    d, L, N, W, lo, hi, seed = wl.systems[0]
    lnW = workloads.random_log_weights(d * N + 1, 3, 0.05)
    launch = BENCH_SHAPES[wl.name] if shape == "bench" else _tuned_shape(wl.systems, [lnW])
    sweeps = 20
    pick = list(range(0, W, 32))
    with m.Mucal(wl.systems, per_walker_hist=True) as mc:
        mc.set_launch(**launch)
        mc.set_weights(0, lnW)
        mc.run_iteration(sweeps, 0)
        H, per = mc.histogram(0, per_walker=True)
        assert H.sum() == W * sweeps * N
        np.testing.assert_array_equal(H, per.sum(axis=0))
        S, occ, E = _oracle_states(d, L, N, W, seed, pick)
        T = chain.thresholds(d, -d * N, 0, lnW)
        hist, _ = chain.run_walkers(d, L, N, seed, 0, sweeps * N, -d * N, 0, T, S, occ, E,
                                    walkers=pick)
        np.testing.assert_array_equal(per[pick], hist)
        for i, w in enumerate(pick):
            _assert_walker_equal(mc, 0, w, S[i], occ[i], E[i])


@pytest.mark.parametrize("shape", ["bench", "tuned"])
def test_batched_every_walker_of_two_systems(shape):
    """The 27-system batch in one launch: every walker of its largest system
    (3D L=40, N=6400, 2366 walkers) and of the largest 2D system (L=128,
    N=1638, 606 walkers) bit-exact against the oracle."""
    wl = workloads.batched_uneven()
    lnWs = [workloads.random_log_weights(s[0] * s[2] + 1, 200 + i, scale=0.05)
            for i, s in enumerate(wl.systems)]
    launch = (BENCH_SHAPES[wl.name] if shape == "bench"
              else _tuned_shape(wl.systems, lnWs))
    big3 = max(range(len(wl.systems)), key=lambda i: (wl.systems[i][0] == 3, wl.systems[i][2]))
    big2 = max(range(len(wl.systems)), key=lambda i: (wl.systems[i][0] == 2, wl.systems[i][2]))
    _every_walker_one_iteration(wl.systems, [big3, big2], 5, 7, launch, lnWs)


# ------------------------------------------ threshold-row window (mode 2) ---
# Each walker keeps 32 rows of the threshold table around its energy in
# shared memory and refills them with bulk copies as the energy moves; the
# chain must stay the oracle's.  thr_window = 2 forces the windows even where
# the table would fit in shared memory, so small systems exercise them: few
# bins (the window holds the whole table), walkers at the window's ends,
# strongly sloped weights (energies run far, many refills), every lane count,
# both views, persistent and tunnelling flavours.

WINDOW_LAUNCHES = [
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=2, walkers_per_block=16, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4, walkers_per_block=24, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1,
         persistent=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=32, walkers_per_block=3, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=4, walkers_per_block=8, bits_in_smem=1,
         persistent=1),
]


@pytest.mark.parametrize("launch", WINDOW_LAUNCHES, ids=_lid)
@pytest.mark.parametrize("desc,sweeps,slope", [
    ((2, 8, 6, 21, 0, 0, 4), 60, 0.0),         # 13 bins: the window covers the whole table
    ((2, 24, 80, 37, 0, 0, 8), 40, -1.5),      # 161 bins, weights favour low E: runs down
    ((3, 10, 150, 29, 0, 0, 12), 15, 0.8),     # 3D, 451 bins, weights favour high E
    ((2, 40, 300, 19, -450, -30, 16), 20, 0.3),  # user window, walkers near its top
])
def test_threshold_window_bit_exact(desc, sweeps, slope, launch):
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = _window(d, N, lo, hi)
    nb = e_hi - e_lo + 1
    S, occ, E = _oracle_states(d, L, N, W, seed)
    if lo or hi:
        ok = (E >= e_lo) & (E <= e_hi)
        if not ok.all():
            pytest.skip("a random placement lies outside the user window")
    lnW = workloads.random_log_weights(nb, 7, scale=0.3) + slope * np.arange(nb)
    lnW -= lnW.max()
    with m.Mucal([desc], per_walker_hist=True) as mc:
        mc.set_launch(**dict(launch, thr_window=2))
        assert mc.launch()["thr_window"] == 2
        mc.set_weights(0, lnW)
        T = chain.thresholds(d, e_lo, e_hi, lnW)
        for it in range(3):
            mc.run_iteration(sweeps, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            H, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
        for w in range(W):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])


def test_threshold_window_tunnel_flavour_bit_exact():
    d, L, N, W, seed = 2, 20, 60, 24, 31
    nb = d * N + 1
    lnW = workloads.random_log_weights(nb, 3, 0.6)
    S, occ, E = _oracle_states(d, L, N, W, seed)
    T = chain.thresholds(d, -d * N, 0, lnW)
    tstate = np.zeros(W, np.uint8)
    tcount = np.zeros(W, np.int64)
    with m.Mucal([(d, L, N, W, 0, 0, seed)], per_walker_hist=True) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=8,
                      bits_in_smem=1, thr_window=2)
        mc.set_weights(0, lnW)
        mc.set_tunnel_window(0, -60, -20)
        for it in range(2):
            mc.run_iteration(50, it)
            hist = chain.run_walkers_tunnel(d, L, N, seed, it, 50 * N, -d * N, 0, T, S, occ, E,
                                            -60, -20, tstate, tcount)
            _, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
        total, per_w, st = mc.tunnel_counts(0)
        np.testing.assert_array_equal(per_w.astype(np.int64), tcount)
        np.testing.assert_array_equal(st, tstate)


def test_window_setting_falls_back_when_it_does_not_fit():
    """3D L=32 with 56 walkers per block: the bitsets fill shared memory, the
    windows cannot join them, the launch reads thresholds from global memory
    and reports it; with fewer walkers per block the windows are used."""
    with m.Mucal([(3, 32, 3277, 64, 0, 0, 0)]) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4, walkers_per_block=56,
                      bits_in_smem=1, thr_window=1)
        assert mc.launch()["thr_window"] == 0
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4, walkers_per_block=32,
                      bits_in_smem=1, thr_window=1)
        assert mc.launch()["thr_window"] == 1


# ------------------------------------------------- multi-commit rounds ------
# One round may commit several accepted moves in attempt order (a later lane
# re-decides at the energy its predecessors reached while its own energy
# change still holds).  The chain must stay the one-thread chain: every lane
# count that has the rounds, both views, bitsets in shared or global memory,
# persistent launches, thresholds staged in shared memory (small tables) and
# read from global memory (the full-size launches below), and weights that
# make nearly every move accepted (lnW = 0: many commits per round) as well as
# sloped ones (long runs, energies moving several rows in one round).

MC_LAUNCHES = [
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=4, walkers_per_block=24, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1,
         persistent=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=32, walkers_per_block=3, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=4, walkers_per_block=8, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=16, walkers_per_block=2, bits_in_smem=1,
         persistent=1),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=32, walkers_per_block=1, bits_in_smem=1),
]


@pytest.mark.parametrize("launch", MC_LAUNCHES, ids=_lid)
@pytest.mark.parametrize("desc,sweeps,slope,scale", [
    ((2, 16, 32, 40, 0, 0, 0), 200, None, 0.0),     # lnW = 0: every move with dE <= 0 taken
    ((2, 24, 80, 37, 0, 0, 8), 40, -1.5, 0.3),      # weights favour low E: runs down
    ((3, 10, 150, 29, 0, 0, 12), 15, 0.8, 0.3),     # 3D, weights favour high E
    ((3, 6, 170, 21, 0, 0, 5), 30, 0.0, 1.0),       # 3D dense (rho 0.79): neighbourhoods overlap
    ((2, 40, 300, 19, -450, -30, 16), 20, 0.3, 0.3),  # user window, walkers near its top
    ((2, 8, 3, 9, 0, 0, 3), 7, 0.0, 0.5),           # 21 attempts per walker: ragged batches
    ((2, 3, 1, 5, 0, 0, 77), 200, 0.0, 0.5),        # one particle on 3 x 3
    ((3, 5, 124, 4, 0, 0, 9), 20, 0.0, 0.5),        # one hole
])
def test_multi_commit_bit_exact(desc, sweeps, slope, scale, launch):
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = _window(d, N, lo, hi)
    nb = e_hi - e_lo + 1
    S, occ, E = _oracle_states(d, L, N, W, seed)
    if lo or hi:
        if not ((E >= e_lo) & (E <= e_hi)).all():
            pytest.skip("a random placement lies outside the user window")
    if slope is None:
        lnW = np.zeros(nb)
    else:
        lnW = workloads.random_log_weights(nb, 7, scale=scale) + slope * np.arange(nb)
        lnW -= lnW.max()
    with m.Mucal([desc], per_walker_hist=True) as mc:
        try:
            mc.set_launch(**dict(launch, multi_commit=1))
        except m.MucalError:
            # the fields of the block's walkers do not fit: one walker per block
            mc.set_launch(**dict(launch, lanes_per_walker=32, walkers_per_block=1,
                                 multi_commit=1))
        assert mc.launch()["multi_commit"] == 1
        mc.set_weights(0, lnW)
        T = chain.thresholds(d, e_lo, e_hi, lnW)
        for it in range(3):
            mc.run_iteration(sweeps, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            H, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
            np.testing.assert_array_equal(H, hist.sum(axis=0))
        acc = mc.stats(0)
        for w in range(W):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])
        assert acc["attempts"] == W * sweeps * N


def test_multi_commit_uint32_lists_bit_exact():
    """V = 66049 > 65536 sites: 32-bit list entries (two shuffles per pair)."""
    desc = (2, 257, 300, 3, 0, 0, 5)
    d, L, N, W, lo, hi, seed = desc
    nb = d * N + 1
    lnW = workloads.random_log_weights(nb, 2, scale=0.3)
    S, occ, E = _oracle_states(d, L, N, W, seed)
    with m.Mucal([desc], per_walker_hist=True) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=4,
                      bits_in_smem=0, multi_commit=1)
        mc.set_weights(0, lnW)
        T = chain.thresholds(d, -d * N, 0, lnW)
        for it in range(2):
            mc.run_iteration(10, it)
            hist, _ = chain.run_walkers(d, L, N, seed, it, 10 * N, -d * N, 0, T, S, occ, E)
            _, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
        for w in range(W):
            _assert_walker_equal(mc, 0, w, S[w], occ[w], E[w])


def test_multi_commit_reported_only_where_it_applies():
    with m.Mucal([(2, 16, 32, 64, 0, 0, 0)]) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=2, walkers_per_block=16,
                      bits_in_smem=1, multi_commit=1)
        assert mc.launch()["multi_commit"] == 0          # 2 lanes: one-commit rounds
        mc.set_launch(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=32,
                      bits_in_smem=1, multi_commit=1)
        assert mc.launch()["multi_commit"] == 0
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=8,
                      bits_in_smem=1, thr_window=2, multi_commit=1)
        assert mc.launch()["multi_commit"] == 0          # row windows: one-commit rounds
        assert mc.launch()["thr_window"] == 2
        mc.set_launch(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=8,
                      bits_in_smem=1, multi_commit=1)
        assert mc.launch()["multi_commit"] == 1
        with pytest.raises(m.MucalError):
            mc.set_launch(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=8,
                          bits_in_smem=1, multi_commit=2)


def test_multi_commit_tunnel_flavour_runs_one_commit_rounds():
    """With tunnelling events recorded the one-commit rounds run; the chain and
    the events are the oracle's."""
    d, L, N, W, seed = 2, 20, 60, 24, 31
    nb = d * N + 1
    lnW = workloads.random_log_weights(nb, 3, 0.6)
    S, occ, E = _oracle_states(d, L, N, W, seed)
    T = chain.thresholds(d, -d * N, 0, lnW)
    tstate = np.zeros(W, np.uint8)
    tcount = np.zeros(W, np.int64)
    with m.Mucal([(d, L, N, W, 0, 0, seed)], per_walker_hist=True) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=8,
                      bits_in_smem=1, multi_commit=1)
        mc.set_weights(0, lnW)
        mc.set_tunnel_window(0, -60, -20)
        for it in range(2):
            mc.run_iteration(50, it)
            hist = chain.run_walkers_tunnel(d, L, N, seed, it, 50 * N, -d * N, 0, T, S, occ, E,
                                            -60, -20, tstate, tcount)
            _, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
        total, per_w, st = mc.tunnel_counts(0)
        np.testing.assert_array_equal(per_w.astype(np.int64), tcount)


@pytest.mark.parametrize("wl_name", ["3d-L32-N3277-w8192", "batched-27-systems-w16384"])
def test_multi_commit_full_size_global_thresholds(wl_name):
    """The benchmark shapes with multi-commit rounds: thresholds read from
    global memory (the tables do not fit beside the bitsets), sampled walkers
    of every system against the oracle, sum H counts every attempt."""
    if wl_name.startswith("batched"):
        wl = workloads.batched_uneven()
    else:
        wl = workloads.LARGE_3D
    launch = dict(BENCH_SHAPES[wl_name], thr_window=0, multi_commit=1)
    lnWs = [workloads.random_log_weights(s[0] * s[2] + 1, 300 + i, scale=0.05)
            for i, s in enumerate(wl.systems)]
    sweeps, it = 5, 3
    with m.Mucal(wl.systems) as mc:
        mc.set_launch(**launch)
        cfg = mc.launch()
        assert cfg["multi_commit"] == 1 and cfg["thr_window"] == 0
        for i, lnW in enumerate(lnWs):
            mc.set_weights(i, lnW)
        mc.run_iteration(sweeps, it)
        for i, (d, L, N, W, lo, hi, seed) in enumerate(wl.systems):
            H = mc.histogram(i)
            assert H.sum() == W * sweeps * N
            pick = sorted({0, W // 3, W - 1})
            S, occ, E = _oracle_states(d, L, N, W, seed, pick)
            T = chain.thresholds(d, -d * N, 0, lnWs[i])
            chain.run_walkers(d, L, N, seed, it, sweeps * N, -d * N, 0, T, S, occ, E, walkers=pick)
            for q, w in enumerate(pick):
                _assert_walker_equal(mc, i, w, S[q], occ[q], E[q])
