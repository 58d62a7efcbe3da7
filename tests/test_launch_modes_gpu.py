"""Persistent launches and CUDA-graph iterations give the same chains.

A persistent launch runs only the blocks that fit on the device and lets
them pull blocks of walkers from a counter; graph mode replays one captured
iteration with the iteration number updated.  Both must leave every walker's
chain unchanged: every histogram bit-exact with the oracle."""
import numpy as np
import pytest

from oracle import chain
from oracle.recursion import recursive_update
from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import workloads

pytestmark = pytest.mark.gpu

GROUP8P = dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=4,
               bits_in_smem=1, persistent=1)
THREADP = dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=7,
               bits_in_smem=0, persistent=1)
GROUP8 = dict(GROUP8P, persistent=0)
FIELD8P = dict(GROUP8P, kernel=m.MUCAL_KERNEL_FIELD)
GROUP8MC = dict(GROUP8, multi_commit=1)
FIELD8PMC = dict(FIELD8P, multi_commit=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


@pytest.mark.parametrize("launch,graph", [(GROUP8P, False), (GROUP8P, True), (THREADP, True),
                                          (GROUP8, True), (FIELD8P, False), (FIELD8P, True),
                                          (GROUP8MC, True), (FIELD8PMC, True)],
                         ids=["G8-persistent", "G8-persistent-graph", "thread-persistent-graph",
                              "G8-graph", "field-G8-persistent", "field-G8-persistent-graph",
                              "G8-multi-commit-graph", "field-G8-persistent-multi-commit-graph"])
def test_small_2d_iterations_bit_exact(launch, graph):
    """2D L=16, N=32, 64 walkers (16 blocks of 4 walkers, or 10 blocks of 7
    for the thread kernel), 6 iterations of 500 sweeps with the recursion."""
    d, L, N, W, lo, hi, seed = workloads.SMALL_2D.systems[0]
    e_lo, e_hi = -d * N, 0
    nb = e_hi - e_lo + 1
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    lnW = np.zeros(nb)
    s_cum = np.zeros(nb, bool)
    phat = np.zeros(nb)
    with m.Mucal(workloads.SMALL_2D.systems, per_walker_hist=True) as mc:
        mc.set_launch(**launch)
        assert mc.launch()["persistent"] == launch["persistent"]
        mc.set_graph_mode(graph)
        for it in range(6):
            T = chain.thresholds(d, e_lo, e_hi, lnW)
            mc.run_iteration(500, 7 * it + 1)
            hist, _ = chain.run_walkers(d, L, N, seed, 7 * it + 1, 500 * N, e_lo, e_hi, T, S, occ, E)
            H, per = mc.histogram(0, per_walker=True)
            np.testing.assert_array_equal(per, hist)
            g_lnW, _ = mc.update_weights(0, m.MUCAL_SCHEME_RECURSIVE)
            lnW, s_cum, phat = recursive_update(lnW, hist.sum(axis=0), s_cum, phat)
            np.testing.assert_allclose(g_lnW, lnW, rtol=1e-12, atol=1e-12 * max(1, np.abs(lnW).max()))
        st = mc.stats(0)
        assert st["attempts"] == W * 500 * N and st["kernel_ms"] > 0


def test_graph_recaptures_on_changes():
    """Graph mode across a change of sweeps, of launch shape, of the rounds
    (multi-commit on and off) and of the kernel flavour (tunnelling switched
    on): every iteration still equals the oracle."""
    desc = (3, 6, 40, 21, 0, 0, 40)
    d, L, N, W, lo, hi, seed = desc
    nb = d * N + 1
    lnW = workloads.random_log_weights(nb, 3, scale=0.3)
    T = chain.thresholds(d, -d * N, 0, lnW)
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    st = np.zeros(W, np.uint8)
    cnt = np.zeros(W, np.int64)
    plan = [(20, GROUP8, False), (20, GROUP8, False), (35, GROUP8, False), (35, GROUP8MC, False),
            (35, GROUP8, False), (35, GROUP8P, False), (35, GROUP8P, True), (10, THREADP, True)]
    with m.Mucal([desc], per_walker_hist=True) as mc:
        mc.set_weights(0, lnW)
        mc.set_graph_mode(True)
        for it, (sweeps, launch, tun) in enumerate(plan):
            mc.set_launch(**launch)
            if tun and it == 6:
                mc.set_tunnel_window(0, -60, -20)
            mc.run_iteration(sweeps, it)
            if tun:
                hist = chain.run_walkers_tunnel(d, L, N, seed, it, sweeps * N, -d * N, 0, T, S, occ,
                                                E, -60, -20, st, cnt)
            else:
                hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, -d * N, 0, T, S, occ, E)
            np.testing.assert_array_equal(mc.histogram(0, per_walker=True)[1], hist)
        total, g_cnt, g_st = mc.tunnel_counts(0)
        np.testing.assert_array_equal(g_cnt.astype(np.int64), cnt)
        np.testing.assert_array_equal(g_st, st)


def test_persistent_batched_full_size_sampled():
    """The 27-system batched workload (16 384 walkers) in one persistent,
    graph-captured launch: the summed histograms account for every attempt
    and sampled walkers of three systems equal the oracle."""
    wl = workloads.batched_uneven()
    sweeps = 3
    with m.Mucal(wl.systems, per_walker_hist=True) as mc:
        mc.set_launch(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=16, walkers_per_block=8,
                      bits_in_smem=1, persistent=1)
        mc.set_graph_mode(True)
        mc.run_iteration(sweeps, 0)
        mc.run_iteration(sweeps, 1)
        for i in (0, 13, len(wl.systems) - 1):
            d, L, N, W, lo, hi, seed = wl.systems[i]
            H, per = mc.histogram(i, per_walker=True)
            assert H.sum() == W * sweeps * N
            pick = sorted({0, W // 2, W - 1})
            S, occ, E = chain.init_walkers(d, L, N, W, seed)
            S, occ, E = S[pick].copy(), occ[pick].copy(), E[pick].copy()
            T = chain.thresholds(d, -d * N, 0, np.zeros(d * N + 1))
            for it in range(2):
                hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, -d * N, 0, T, S, occ, E,
                                            walkers=pick)
            np.testing.assert_array_equal(per[pick], hist)


def test_default_launch_is_field_kernel_where_fields_fit():
    """The library's default launch is the field kernel when every system's
    neighbour-count fields fit into shared memory at 16 walkers per block
    (2D L=64: 4 KB per walker), else the group kernel (3D L=32: 32 KB)."""
    with m.Mucal([(2, 64, 410, 64, 0, 0, 0)]) as mc:
        assert mc.launch()["kernel"] == m.MUCAL_KERNEL_FIELD
    with m.Mucal([(3, 32, 3277, 64, 0, 0, 0)]) as mc:
        assert mc.launch()["kernel"] == m.MUCAL_KERNEL_GROUP
    with m.Mucal([(2, 16, 32, 8, 0, 0, 0), (3, 32, 3277, 8, 0, 0, 1)]) as mc:
        assert mc.launch()["kernel"] == m.MUCAL_KERNEL_GROUP
