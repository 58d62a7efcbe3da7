"""numpy front end of the C oracle (test infrastructure only).

Each function is a thin call into ``mucal_oracle.c``; the arithmetic lives
there.  Walker states are kept as plain arrays:

* ``S``   int32[n_walkers, V]: S[:, :N] particle sites, S[:, N:] empty sites;
* ``occ`` uint8[n_walkers, V]: occupation n_i (Sec. 3);
* ``E``   int64[n_walkers]: energy of Eq. 5 (J = 1).
"""
from __future__ import annotations

import numpy as np

from .build import load_oracle


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def volume(d: int, L: int) -> int:
    return int(L) ** int(d)


def philox(counters: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """Philox4x32-10 blocks: counters uint32[n,4], keys uint32[n,2] -> uint32[n,4]."""
    lib = load_oracle()
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(keys, dtype=np.uint32).reshape(-1, 2)
    assert c.shape[0] == k.shape[0]
    out = np.zeros_like(c)
    lib.orc_philox_batch(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


def neighbours(d: int, L: int, s: int) -> np.ndarray:
    lib = load_oracle()
    nb = np.zeros(6, dtype=np.int64)
    lib.orc_neighbours(d, L, int(s), _ptr(nb))
    return nb[: 2 * d].copy()


def energy(d: int, L: int, occ: np.ndarray) -> int:
    """Eq. 5 with J = 1 for one occupation array."""
    lib = load_oracle()
    o = np.ascontiguousarray(occ, dtype=np.uint8)
    assert o.size == volume(d, L)
    return int(lib.orc_energy(d, L, _ptr(o)))


def delta_e(d: int, L: int, occ: np.ndarray, a: int, b: int) -> int:
    lib = load_oracle()
    o = np.ascontiguousarray(occ, dtype=np.uint8)
    return int(lib.orc_delta_e(d, L, _ptr(o), int(a), int(b)))


def init_walkers(d: int, L: int, N: int, n_walkers: int, seed_base: int):
    """Initial placement of every walker (walker w uses seed seed_base + w)."""
    lib = load_oracle()
    V = volume(d, L)
    S = np.zeros((n_walkers, V), dtype=np.int32)
    occ = np.zeros((n_walkers, V), dtype=np.uint8)
    E = np.zeros(n_walkers, dtype=np.int64)
    lib.orc_init_walkers(d, L, N, n_walkers, np.uint64(seed_base), _ptr(S), _ptr(occ), _ptr(E))
    return S, occ, E


def thresholds(d: int, e_lo: int, e_hi: int, lnW: np.ndarray) -> np.ndarray:
    """uint32[n_bins, 4d+1] acceptance thresholds from float64 lnW (Sec. 2)."""
    lib = load_oracle()
    w = np.ascontiguousarray(lnW, dtype=np.float64)
    nb = e_hi - e_lo + 1
    assert w.size == nb
    T = np.zeros((nb, 4 * d + 1), dtype=np.uint32)
    lib.orc_thresholds(d, e_lo, e_hi, _ptr(w), _ptr(T))
    return T


def run_walkers(d: int, L: int, N: int, seed_base: int, iteration: int, n_attempts: int,
                e_lo: int, e_hi: int, T: np.ndarray, S: np.ndarray, occ: np.ndarray,
                E: np.ndarray, walkers=None):
    """Advance walkers in place by ``n_attempts`` attempts each (Sec. 2).

    ``walkers`` optionally selects a subset (walker ids, for seeds); the state
    arrays then hold only those walkers, in that order.  Returns
    (hist int64[n, n_bins], accepts int64[n]).
    """
    lib = load_oracle()
    n = S.shape[0]
    nb = e_hi - e_lo + 1
    hist = np.zeros((n, nb), dtype=np.int64)
    acc = np.zeros(n, dtype=np.int64)
    Tc = np.ascontiguousarray(T, dtype=np.uint32)
    assert S.dtype == np.int32 and occ.dtype == np.uint8 and E.dtype == np.int64
    if walkers is None:
        bad = lib.orc_run_walkers(d, L, N, n, np.uint64(seed_base), np.uint32(iteration),
                                  int(n_attempts), e_lo, e_hi, _ptr(Tc), _ptr(S), _ptr(occ),
                                  _ptr(E), _ptr(hist), _ptr(acc))
        if bad:
            raise ValueError(f"{bad} walkers outside the energy window")
        return hist, acc
    V = volume(d, L)
    for i, w in enumerate(walkers):
        Si = S[i]
        oi = occ[i]
        Ei = E[i: i + 1]
        hi = hist[i]
        ai = acc[i: i + 1]
        rc = lib.orc_run_walker(d, L, N, np.uint64(seed_base + int(w)), np.uint32(iteration),
                                int(n_attempts), e_lo, e_hi, _ptr(Tc), _ptr(Si), _ptr(oi),
                                _ptr(Ei), _ptr(hi), _ptr(ai))
        if rc != 0:
            raise ValueError(f"walker {w} outside the energy window")
        assert Si.size == V
    return hist, acc


def run_walkers_tunnel(d: int, L: int, N: int, seed_base: int, iteration: int, n_attempts: int,
                       e_lo: int, e_hi: int, T: np.ndarray, S: np.ndarray, occ: np.ndarray,
                       E: np.ndarray, t_min: int, t_max: int, tstate: np.ndarray,
                       tcount: np.ndarray) -> np.ndarray:
    """run_walkers with per-walker tunnelling bookkeeping (Sec. 4): tstate
    uint8[n] (0 none, 1 low end last, 2 high end last) and tcount int64[n]
    are updated in place.  Returns hist int64[n, n_bins]."""
    lib = load_oracle()
    n = S.shape[0]
    hist = np.zeros((n, e_hi - e_lo + 1), dtype=np.int64)
    Tc = np.ascontiguousarray(T, dtype=np.uint32)
    assert tstate.dtype == np.uint8 and tcount.dtype == np.int64
    bad = lib.orc_run_walkers_tunnel(d, L, N, n, np.uint64(seed_base), np.uint32(iteration),
                                     int(n_attempts), e_lo, e_hi, _ptr(Tc), _ptr(S), _ptr(occ),
                                     _ptr(E), _ptr(hist), int(t_min), int(t_max), _ptr(tstate),
                                     _ptr(tcount))
    if bad:
        raise ValueError(f"{bad} walkers outside the energy window")
    return hist


def enumerate_omega(d: int, L: int, N: int) -> dict:
    """Exact Omega(E) by visiting all C(V, N) configurations (V <= 64)."""
    lib = load_oracle()
    om = np.zeros(d * N + 1, dtype=np.int64)
    cnt = lib.orc_enumerate(d, L, N, _ptr(om))
    if cnt < 0:
        raise ValueError("enumeration needs V <= 64")
    return {-e: int(om[e]) for e in range(d * N + 1) if om[e] > 0}


def energy_mask(d: int, L: int, mask: int) -> int:
    return int(load_oracle().orc_energy_mask(d, L, np.uint64(mask)))


def delta_e_mask(d: int, L: int, mask: int, a: int, b: int) -> int:
    return int(load_oracle().orc_delta_e_mask(d, L, np.uint64(mask), int(a), int(b)))


def ising_fixed_m(d: int, L: int, n_up: int, seed: int, beta_ising: float,
                  n_attempts: int, n_discard: int):
    """Fixed-magnetisation Metropolis Ising run (Sec. 4): returns (<H^I>, <(H^I)^2>)."""
    import ctypes
    lib = load_oracle()
    me = ctypes.c_double()
    me2 = ctypes.c_double()
    rc = lib.orc_ising_fixed_m(d, L, n_up, np.uint64(seed), float(beta_ising), int(n_attempts),
                               int(n_discard), ctypes.addressof(me), ctypes.addressof(me2))
    if rc != 0:
        raise MemoryError
    return me.value, me2.value


def largest_droplet(d: int, L: int, occ: np.ndarray) -> int:
    """Particles in the largest nearest-neighbour cluster (Sec. 3), periodic."""
    o = np.ascontiguousarray(occ, dtype=np.uint8).reshape(-1)
    assert o.size == volume(d, L)
    return int(load_oracle().orc_largest_cluster(d, L, _ptr(o)))


def replica_exchange(beta, seeds, round_: int, parity: int, S: np.ndarray, occ: np.ndarray,
                     E: np.ndarray) -> np.ndarray:
    """Parallel-tempering exchange between neighbouring systems, in place on
    S[K, W, V], occ[K, W, V], E[K, W]; returns accepted exchanges per pair."""
    K, W, V = S.shape
    b = np.ascontiguousarray(beta, dtype=np.float64)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    assert b.size == K and sd.size == K
    assert S.dtype == np.int32 and occ.dtype == np.uint8 and E.dtype == np.int64
    acc = np.zeros(max(K - 1, 1), dtype=np.int64)
    load_oracle().orc_replica_exchange(K, W, V, _ptr(sd), _ptr(b), np.uint32(round_), int(parity),
                                       _ptr(S), _ptr(occ), _ptr(E), _ptr(acc))
    return acc[: K - 1]


def num_threads() -> int:
    return int(load_oracle().orc_num_threads())
