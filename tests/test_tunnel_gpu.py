"""GPU parity of the tunnelling count (Sec. 4): per-walker events and last
ends after several iterations, bit-exact with the oracle's chain, in every
launch shape of the parity tests."""
import numpy as np
import pytest

from oracle import chain
from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import workloads

pytestmark = pytest.mark.gpu

LAUNCHES = [
    dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=32, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1, walkers_per_block=7, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=2, walkers_per_block=16, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
    dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=32, walkers_per_block=5, bits_in_smem=0),
    dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=8, walkers_per_block=12, bits_in_smem=1),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


def _ideal_weights(d, L, N):
    omega = chain.enumerate_omega(d, L, N)
    return np.array([-np.log(omega[e]) if e in omega else 0.0 for e in range(-d * N, 1)])


def _compare(desc, lnW, ends, sweeps, iters, launch=None, set_ends=True):
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = (-d * N, 0) if lo == 0 and hi == 0 else (lo, hi)
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    st = np.zeros(W, np.uint8)
    cnt = np.zeros(W, np.int64)
    with m.Mucal([desc]) as mc:
        if launch:
            mc.set_launch(**launch)
        mc.set_weights(0, lnW)
        mc.set_tunnel_window(0, *(ends if set_ends else (0, 0)))
        for it in range(iters):
            mc.run_iteration(sweeps, it)
            chain.run_walkers_tunnel(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E,
                                     ends[0], ends[1], st, cnt)
        total, g_cnt, g_st = mc.tunnel_counts(0)
    np.testing.assert_array_equal(g_cnt.astype(np.int64), cnt)
    np.testing.assert_array_equal(g_st, st)
    assert total == cnt.sum()
    return total


@pytest.mark.parametrize("launch", LAUNCHES,
                         ids=lambda c: f"k{c['kernel']}-G{c['lanes_per_walker']}-w{c['walkers_per_block']}")
def test_tunnel_counts_bit_exact_4x4(launch):
    """4x4, N = 5 at the ideal weights 1/Omega: walkers travel between
    E = -5 and E = 0 many times per iteration."""
    total = _compare((2, 4, 5, 37, 0, 0, 11), _ideal_weights(2, 4, 5), (-5, 0), 200, 4, launch)
    assert total > 37 * 4


@pytest.mark.parametrize("launch", LAUNCHES[:1] + LAUNCHES[3:4],
                         ids=lambda c: f"k{c['kernel']}-G{c['lanes_per_walker']}")
def test_tunnel_counts_bit_exact_window_defaults(launch):
    """2D L=16, N=32 with random smooth weights and the default ends (the
    window's ends [-64, 0]); and with ends inside the window."""
    lnW = workloads.random_log_weights(65, 4, scale=0.4)
    _compare((2, 16, 32, 64, 0, 0, 0), lnW, (-64, 0), 50, 3, launch, set_ends=False)
    _compare((2, 16, 32, 64, 0, 0, 0), lnW, (-20, -8), 50, 3, launch)


def test_tunnel_counts_full_size_medium_2d():
    """64x64, N = 410, 4096 walkers, window [-820, 0] in the default launch
    shape, lnW = 0: random placements hold about 82 bonds (E = -82 +- 9), so
    ends at -88 and -76 are crossed often."""
    desc = workloads.MEDIUM_2D.systems[0]
    total = _compare(desc, np.zeros(821), (-88, -76), 20, 2)
    assert total > 0


def test_tunnel_window_errors_and_reset():
    with m.Mucal([(2, 8, 10, 4, 0, 0, 0)]) as mc:
        mc.set_weights(0, np.zeros(21))
        mc.run_iteration(100, 0)
        assert mc.tunnel_counts(0)[0] == 0          # bookkeeping is off until switched on
        with pytest.raises(m.MucalError):
            mc.set_tunnel_window(0, -5, -5)
        with pytest.raises(m.MucalError):
            mc.set_tunnel_window(0, -30, 0)
        mc.set_weights(0, np.zeros(21))
        mc.run_iteration(100, 0)
        mc.reset_tunnel_counts()
        total, cnt, st = mc.tunnel_counts(0)
        assert total == 0 and (cnt == 0).all() and (st == 0).all()


def test_scaling_study_runs_to_the_event_criterion():
    """The Fig. 3 study on 4x4, N = 5 (window [-5, 0]): every run reaches 30
    tunnelling events, and the per-walker sweeps follow total / p."""
    from paper_1401_4076_gb300 import scaling
    rows = scaling.study(2, 4, 5, (-5, 0), [1, 8], seeds=2, total_sweeps=64, max_iter=300)
    assert [r["walkers"] for r in rows] == [1, 8]
    for r in rows:
        assert r["converged"] == r["runs"] == 2
    assert rows[0]["sweeps_per_walker"] == pytest.approx(64, rel=0.05)
    assert rows[1]["sweeps_per_walker"] == pytest.approx(8, rel=0.05)
    assert rows[0]["speedup_S_p"] == 1.0
