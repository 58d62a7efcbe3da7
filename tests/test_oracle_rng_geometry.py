"""Pins of the oracle's random numbers, geometry, energy and initial placement.

Each check compares the oracle with something other than itself: Triton's own
Philox implementation, numpy's roll-based neighbour sums, hand-countable
energies, or distributional facts of a uniform random subset.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import chain, muca

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- Philox ----

def test_philox_matches_triton_interpreter(tmp_path):
    """Philox4x32-10 (Salmon et al., SC'11) against Triton's implementation."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(2024)
    n = 512
    c = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    c[0] = 0
    k[0] = 0
    c[1] = [0xFFFFFFFF] * 4
    k[1] = [0xFFFFFFFF] * 2
    np.save(tmp_path / "c.npy", c)
    np.save(tmp_path / "k.npy", k)
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "philox_triton_ref.py"),
                        str(tmp_path / "c.npy"), str(tmp_path / "k.npy"),
                        str(tmp_path / "o.npy")], capture_output=True, text=True, env=env,
                       timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.load(tmp_path / "o.npy")
    np.testing.assert_array_equal(chain.philox(c, k), ref)


def test_philox_counter_sensitivity_and_uniformity():
    """Every counter word and key word changes the output; outputs are uniform."""
    base_c = np.array([[1, 2, 3, 4]], dtype=np.uint32)
    base_k = np.array([[5, 6]], dtype=np.uint32)
    ref = chain.philox(base_c, base_k)[0]
    for i in range(4):
        c = base_c.copy()
        c[0, i] ^= 1
        assert not np.array_equal(chain.philox(c, base_k)[0], ref)
    for i in range(2):
        k = base_k.copy()
        k[0, i] ^= 1
        assert not np.array_equal(chain.philox(base_c, k)[0], ref)
    n = 1 << 16
    c = np.zeros((n, 4), dtype=np.uint32)
    c[:, 0] = np.arange(n, dtype=np.uint32)
    k = np.tile(np.array([[123, 456]], dtype=np.uint32), (n, 1))
    out = chain.philox(c, k).ravel()
    counts = np.bincount(out >> 28, minlength=16)
    exp = out.size / 16
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 45.0          # 15 dof, p ~ 1e-4
    bits = np.unpackbits(out.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.002


# ---------------------------------------------------------------- geometry --

@pytest.mark.parametrize("d,L", [(2, 3), (2, 5), (3, 3), (3, 4)])
def test_neighbours_are_unit_torus_steps(d, L):
    V = L ** d
    shape = (L,) * d
    for s in range(V):
        xs = np.array(np.unravel_index(s, shape[::-1])[::-1])  # x_0 fastest
        nb = chain.neighbours(d, L, s)
        assert len(set(nb.tolist())) == 2 * d
        for t in nb:
            xt = np.array(np.unravel_index(int(t), shape[::-1])[::-1])
            diff = (xt - xs) % L
            nz = np.nonzero(diff)[0]
            assert len(nz) == 1 and diff[nz[0]] in (1, L - 1)
            assert s in chain.neighbours(d, L, int(t)).tolist()


def _roll_energy(d, L, occ):
    """-#occupied nearest-neighbour pairs via numpy.roll on the L^d grid."""
    g = np.asarray(occ, dtype=np.int64).reshape((L,) * d)
    return -int(sum((g * np.roll(g, 1, axis=ax)).sum() for ax in range(d)))


@pytest.mark.parametrize("d,L,N", [(2, 3, 4), (2, 8, 20), (3, 4, 20), (3, 5, 40)])
def test_energy_matches_roll(d, L, N):
    rng = np.random.default_rng(d * 100 + L)
    V = L ** d
    for _ in range(50):
        occ = np.zeros(V, dtype=np.uint8)
        occ[rng.choice(V, N, replace=False)] = 1
        assert chain.energy(d, L, occ) == _roll_energy(d, L, occ)


def test_energy_hand_counted():
    # 4x4: two adjacent full rows wrap around -> 4 + 4 horizontal + 4 vertical = 12 pairs
    occ = np.zeros(16, dtype=np.uint8)
    occ[0:8] = 1
    assert chain.energy(2, 4, occ) == -12
    # checkerboard: no occupied pairs
    cb = np.array([(x + y) % 2 for y in range(4) for x in range(4)], dtype=np.uint8)
    assert chain.energy(2, 4, cb) == 0
    # full 3x3x3 lattice: 3 * 27 bonds
    assert chain.energy(3, 3, np.ones(27, dtype=np.uint8)) == -81


@pytest.mark.parametrize("d,L,N", [(2, 4, 6), (2, 7, 10), (3, 4, 12)])
def test_delta_e_equals_recount(d, L, N):
    """dE of a jump = E(after) - E(before), including a adjacent to b."""
    rng = np.random.default_rng(7 + L)
    V = L ** d
    adjacent_seen = 0
    for _ in range(300):
        occ = np.zeros(V, dtype=np.uint8)
        occ[rng.choice(V, N, replace=False)] = 1
        a = int(rng.choice(np.nonzero(occ)[0]))
        if rng.random() < 0.5:
            cands = [t for t in chain.neighbours(d, L, a) if occ[t] == 0]
            b = int(rng.choice(cands)) if cands else int(rng.choice(np.nonzero(occ == 0)[0]))
        else:
            b = int(rng.choice(np.nonzero(occ == 0)[0]))
        adjacent_seen += b in chain.neighbours(d, L, a)
        after = occ.copy()
        after[a] = 0
        after[b] = 1
        assert chain.delta_e(d, L, occ, a, b) == _roll_energy(d, L, after) - _roll_energy(d, L, occ)
    assert adjacent_seen > 50


# ---------------------------------------------------------- Ising map, Eq. 5 --

@pytest.mark.parametrize("d,L,N", [(2, 4, 5), (2, 6, 17), (3, 4, 30)])
def test_gas_ising_map_exact(d, L, N):
    """H_gas = H_Ising/4 + c(N) for every configuration (Eq. 5), c(N) = d(V/4 - N)."""
    rng = np.random.default_rng(N)
    V = L ** d
    c = muca.ising_constant(d, L, N)
    for _ in range(20):
        occ = np.zeros(V, dtype=np.uint8)
        occ[rng.choice(V, N, replace=False)] = 1
        s = 2 * occ.astype(np.int64) - 1
        g = s.reshape((L,) * d)
        h_ising = -int(sum((g * np.roll(g, 1, axis=ax)).sum() for ax in range(d)))
        assert muca.ising_energy_of_occ(d, L, occ) == h_ising
        assert chain.energy(d, L, occ) == pytest.approx(h_ising / 4.0 + c, abs=1e-12)


# -------------------------------------------------------- initial placement --

def test_init_state_consistent():
    d, L, N = 2, 16, 32
    S, occ, E = chain.init_walkers(d, L, N, 64, 0)
    V = L ** d
    for w in range(64):
        assert sorted(S[w].tolist()) == list(range(V))
        assert occ[w].sum() == N
        assert set(np.nonzero(occ[w])[0].tolist()) == set(S[w, :N].tolist())
        assert E[w] == _roll_energy(d, L, occ[w])
    # different seeds give different placements
    assert len({tuple(sorted(S[w, :N])) for w in range(64)}) == 64


def test_init_uniform_subsets():
    """3x3, N=3: all C(9,3) = 84 subsets equally likely over many seeds."""
    n = 84 * 400
    S, occ, E = chain.init_walkers(2, 3, 3, n, 1000)
    keys = [int(sum(1 << int(s) for s in S[w, :3])) for w in range(n)]
    _, counts = np.unique(keys, return_counts=True)
    assert len(counts) == 84
    exp = n / 84
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 83 + 5 * math.sqrt(2 * 83)
