"""Energy ranges from short parallel-tempering runs (Sec. 3).

The multicanonical runs of Sec. 3 sample the energy range that matters for
the temperatures of interest; the paper finds it with short parallel-
tempering runs at the start of each simulation.  Here a ladder of K copies of
the lattice at canonical weights lnW_k(E) = -beta_k E runs in one context:
every round is one canonical update of all walkers (the library's walker
kernel with those weights) followed by replica exchanges between neighbouring
temperatures (the library's exchange kernel), alternating the pair parity.

The window's lower end is the lowest energy the coldest replicas visit after
a burn-in, minus a margin; its upper end is 0, the largest energy of the
model (an empty-bond gas, which also contains every random initial
placement).  The coldest temperature lies below the target, so the window
covers the condensed side of the target's distribution with room to spare.
"""
from __future__ import annotations

import numpy as np

from . import mucal as m


def ladder(T: float, n_temps: int = 8, cold: float = 0.85, hot: float = 2.0):
    """Inverse temperatures from 1/(cold T) down to 1/(hot T), geometric in
    beta, with 1/T itself on the ladder."""
    b_cold, b_hot = 1.0 / (cold * T), 1.0 / (hot * T)
    betas = np.geomspace(b_cold, b_hot, n_temps)
    j = int(np.argmin(np.abs(betas - 1.0 / T)))
    betas[j] = 1.0 / T
    return betas


def energy_range(d: int, L: int, N: int, T: float, walkers: int = 256, n_temps: int = 8,
                 rounds: int = 200, burn: int = 50, sweeps: int = 5, margin: float = 0.02,
                 seed: int = 0, cuda_stream=None):
    """(e_lo, e_hi, info) for a multicanonical window around temperature T."""
    betas = ladder(T, n_temps)
    e_lo_full = -d * N
    grid = np.arange(e_lo_full, 1, dtype=np.float64)
    systems = [(d, L, N, walkers, 0, 0, seed + k * walkers) for k in range(len(betas))]
    H = np.zeros((len(betas), d * N + 1), dtype=np.int64)
    acc = np.zeros(len(betas) - 1, dtype=np.int64)
    with m.Mucal(systems, cuda_stream=cuda_stream) as mc:
        for k, b in enumerate(betas):
            mc.set_weights(k, -b * grid)
        for r in range(rounds):
            mc.run_iteration(sweeps, r)
            acc += mc.replica_exchange(betas, r, r % 2)
            if r >= burn:
                for k in range(len(betas)):
                    H[k] += mc.histogram(k)
    visited = np.nonzero(H[0])[0]
    cold_min = e_lo_full + int(visited.min())
    j = int(np.argmin(np.abs(betas - 1.0 / T)))
    tv = np.nonzero(H[j])[0]
    pad = max(2, int(round(margin * d * N)))
    lo = max(e_lo_full, cold_min - pad)
    # the energy below which the coldest replicas spent 1 % of their time
    cdf = np.cumsum(H[0]) / max(1, H[0].sum())
    cold_q01 = e_lo_full + int(np.searchsorted(cdf, 0.01))
    info = {"betas": betas.tolist(), "accepted_exchanges": acc.tolist(),
            "cold_q01": cold_q01,
            "hot_max": e_lo_full + int(np.nonzero(H[-1])[0].max()),
            "exchange_proposals_per_pair": (rounds // 2) * walkers,
            "cold_min": cold_min, "target_min": e_lo_full + int(tv.min()),
            "target_max": e_lo_full + int(tv.max())}
    return lo, 0, info
