"""Seeded synthetic workloads (system descriptions and test weight functions).

Shared by the tests, the benchmark and the smoke check for feeding the same
inputs to the CUDA path and to the oracle.  This module holds only workload
shapes and seeded random inputs; none of the method's arithmetic lives here.

The workloads follow the paper's model (Sec. 3): a fixed number N of
particles on a periodic L^d lattice at densities rho = N / V of a few per cent
up to about ten per cent (the paper fixes N and varies L), with many
independent walkers sharing one weight function (Sec. 2).  Walker w of a
system uses seed seed_base + w.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    systems: tuple            # tuples (d, L, N, n_walkers, e_lo, e_hi, seed_base)
    sweeps: int               # sweeps per iteration; one sweep = N attempts
    iterations: int           # iterations of the weight recursion to run
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def attempts_per_iteration(self) -> int:
        return sum(s[3] * s[2] * self.sweeps for s in self.systems)


def n_particles(d: int, L: int, rho: float) -> int:
    return int(round(rho * L ** d))


# 2D L=16, N=32 (rho = 0.125), 64 walkers with seeds 0..63, lnW = 0 start,
# 10 iterations of 2000 sweeps: the small case the oracle runs completely.
SMALL_2D = Workload("2d-L16-N32-w64", ((2, 16, 32, 64, 0, 0, 0),), sweeps=2000, iterations=10)

# 2D L=64, N=410 (rho ~ 0.1), 4096 walkers, full window [-2N, 0].
MEDIUM_2D = Workload("2d-L64-N410-w4096", ((2, 64, 410, 4096, 0, 0, 0),), sweeps=1000,
                     iterations=200)

# 3D L=32, N=3277 (rho ~ 0.1), 8192 walkers, window [-3N, 0].
LARGE_3D = Workload("3d-L32-N3277-w8192", ((3, 32, 3277, 8192, 0, 0, 0),), sweeps=200,
                    iterations=500)


def batched_uneven(total_walkers: int = 16384, seed_base: int = 0) -> Workload:
    """2D L in {32,48,64,96,128} and 3D L in {16,24,32,40}, each at
    rho in {0.02, 0.05, 0.1}; walkers per system proportional to V (largest
    remainder, at least one), summing to total_walkers."""
    shapes = [(2, L) for L in (32, 48, 64, 96, 128)] + [(3, L) for L in (16, 24, 32, 40)]
    rhos = (0.02, 0.05, 0.1)
    combos = [(d, L, rho) for d, L in shapes for rho in rhos]
    vols = np.array([L ** d for d, L, _ in combos], dtype=np.float64)
    quota = total_walkers * vols / vols.sum()
    base = np.maximum(np.floor(quota).astype(np.int64), 1)
    rest = total_walkers - int(base.sum())
    order = np.argsort(-(quota - np.floor(quota)), kind="stable")
    for i in order[:max(rest, 0)]:
        base[i] += 1
    systems = []
    off = seed_base
    for (d, L, rho), w in zip(combos, base):
        systems.append((d, L, n_particles(d, L, rho), int(w), 0, 0, off))
        off += int(w)
    return Workload("batched-27-systems-w%d" % total_walkers, tuple(systems), sweeps=200,
                    iterations=1)


def random_log_weights(n_bins: int, seed: int, scale: float = 0.3) -> np.ndarray:
    """A smooth random walk as test lnW (float64), shifted to max 0."""
    rng = np.random.default_rng(seed)
    w = np.cumsum(rng.normal(scale=scale, size=n_bins))
    return w - w.max()


def mlp_initial_params(seed: int, hidden: int = 128) -> np.ndarray:
    """Seeded fan-in uniform initial parameters of the seeding network, as the
    flat fp32 vector W1[128][4], b1, W2[128][128], b2, W3[128], b3."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape, fan_in in (((hidden, 4), 4), ((hidden,), 4), ((hidden, hidden), hidden),
                          ((hidden,), hidden), ((1, hidden), hidden), ((1,), hidden)):
        lim = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, size=shape).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def mlp_test_batch(n: int, seed: int):
    """Seeded feature rows (4 columns, a few units wide) and smooth targets."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.5, 1.5, size=(n, 4)).astype(np.float32)
    t = (np.sin(X[:, 0]) * X[:, 1] + 0.5 * X[:, 2] ** 2 - 0.3 * X[:, 3]).astype(np.float32)
    return X, t
