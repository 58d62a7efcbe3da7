"""GPU parity of the replica exchange (parallel tempering, Sec. 3): every
walker of every temperature after each round of canonical sweeps and
exchanges, and the accepted exchanges per pair, bit-exact with the oracle."""
import numpy as np
import pytest

from oracle import chain
from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import tempering

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


@pytest.mark.parametrize("d,L,N,W,betas,rounds,sweeps", [
    (2, 8, 12, 32, [0.3, 0.8, 1.3, 2.0], 12, 2),
    (3, 5, 20, 17, [0.5, 0.9, 1.4, 2.2, 3.5], 9, 1),        # odd ladder, ragged walkers
    (2, 257, 300, 3, [1.0, 2.5], 2, 1),                      # uint32 site lists
])
def test_replica_exchange_bit_exact(d, L, N, W, betas, rounds, sweeps):
    K = len(betas)
    V = L ** d
    e_lo = -d * N
    seeds = np.array([1000 + 97 * k * W for k in range(K)], dtype=np.uint64)
    descs = [(d, L, N, W, 0, 0, int(seeds[k])) for k in range(K)]
    lnW = [-b * np.arange(e_lo, 1, dtype=np.float64) for b in betas]
    S = np.zeros((K, W, V), np.int32)
    occ = np.zeros((K, W, V), np.uint8)
    E = np.zeros((K, W), np.int64)
    for k in range(K):
        S[k], occ[k], E[k] = chain.init_walkers(d, L, N, W, int(seeds[k]))
    T = [chain.thresholds(d, e_lo, 0, w) for w in lnW]
    with m.Mucal(descs) as mc:
        for k in range(K):
            mc.set_weights(k, lnW[k])
        for r in range(rounds):
            mc.run_iteration(sweeps, r)
            got = mc.replica_exchange(betas, r, r % 2)
            for k in range(K):
                chain.run_walkers(d, L, N, int(seeds[k]), r, sweeps * N, e_lo, 0, T[k], S[k], occ[k], E[k])
            want = chain.replica_exchange(betas, seeds, r, r % 2, S, occ, E)
            np.testing.assert_array_equal(got, want)
        for k in range(K):
            for w in range(W):
                g_occ, g_S, g_E = mc.walker_state(k, w)
                np.testing.assert_array_equal(g_occ, occ[k, w])
                np.testing.assert_array_equal(g_S, S[k, w])
                assert g_E == E[k, w]


def test_replica_exchange_rejects_bad_ladders():
    with m.Mucal([(2, 8, 12, 4, 0, 0, 0), (2, 8, 13, 4, 0, 0, 9)]) as mc:
        with pytest.raises(m.MucalError):
            mc.replica_exchange([1.0, 2.0], 0, 0)            # N differs
    with m.Mucal([(2, 8, 12, 4, 0, 0, 0), (2, 8, 12, 4, 0, 0, 9)]) as mc:
        with pytest.raises(m.MucalError):
            mc.replica_exchange([1.0, 2.0], 0, 2)
        with pytest.raises(m.MucalError):
            mc.replica_exchange([1.0, 2.0, 3.0], 0, 0)
        with pytest.raises(m.MucalError):
            mc.replica_exchange([1.0, float("nan")], 0, 0)
        assert mc.replica_exchange([1.0, 2.0], 0, 1).tolist() == [0]


def test_energy_range_brackets_the_canonical_distribution():
    """The range finder's window contains every energy the canonical walkers
    at the target temperature visit, and stops above the ground state of a
    condensing 2D system."""
    d, L, N = 2, 40, 60
    lo, hi, info = tempering.energy_range(d, L, N, T=0.375, walkers=256, rounds=150, seed=5)
    assert hi == 0 and lo < info["target_min"] <= info["target_max"] <= 0
    assert lo >= -d * N
