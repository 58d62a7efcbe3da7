"""Parallel multicanonical iteration, exact transition matrix, reweighting.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import chain
from .recursion import extrapolate_edges, flatness, recursive_update, simple_update


class System:
    """One lattice-gas system with its walkers, weights and recursion memory."""

    def __init__(self, d, L, N, n_walkers, seed_base, e_lo=None, e_hi=None):
        self.d, self.L, self.N = int(d), int(L), int(N)
        self.V = chain.volume(d, L)
        self.n_walkers = int(n_walkers)
        self.seed_base = int(seed_base)
        self.e_lo = -self.d * self.N if e_lo is None else int(e_lo)
        self.e_hi = 0 if e_hi is None else int(e_hi)
        self.n_bins = self.e_hi - self.e_lo + 1
        self.S, self.occ, self.E = chain.init_walkers(d, L, N, n_walkers, seed_base)
        self.lnW = np.zeros(self.n_bins)
        self.s_cum = np.zeros(self.n_bins, dtype=bool)
        self.phat = np.zeros(self.n_bins)

    def iterate(self, sweeps, iteration):
        """One iteration of Sec. 2: all walkers run sweeps*N attempts with fixed
        W; returns (H summed by Eq. 2, per-walker histograms, accepts)."""
        T = chain.thresholds(self.d, self.e_lo, self.e_hi, self.lnW)
        hist, acc = chain.run_walkers(self.d, self.L, self.N, self.seed_base, iteration,
                                      int(sweeps) * self.N, self.e_lo, self.e_hi, T,
                                      self.S, self.occ, self.E)
        H = hist.sum(axis=0)
        return H, hist, acc

    def update(self, H, scheme="recursive", t_lo=None, t_hi=None, extrapolate=False):
        if scheme == "simple":
            self.s_cum = self.s_cum | (H > 0)
            self.lnW = simple_update(self.lnW, H)
        else:
            self.lnW, self.s_cum, self.phat = recursive_update(self.lnW, H, self.s_cum, self.phat)
        if extrapolate:
            self.lnW = extrapolate_edges(self.lnW, self.s_cum)
        tl = None if t_lo is None else t_lo - self.e_lo
        th = None if t_hi is None else t_hi - self.e_lo
        return flatness(H, self.s_cum, tl, th)


def run_to_flat(system: System, sweeps, max_iter, scheme="recursive", t_lo=None, t_hi=None,
                goal=0.5, extrapolate=False):
    """Iterate until flatness >= goal; returns (iterations used, last H, flatness)."""
    H = None
    f = -1.0
    for it in range(max_iter):
        H, _, _ = system.iterate(sweeps, it)
        f = system.update(H, scheme, t_lo, t_hi, extrapolate)
        if f >= goal:
            return it + 1, H, f
    return max_iter, H, f


def transition_matrix(d, L, N, T, e_lo):
    """Exact transition matrix of the jump-move chain on occupation sets (V <= 64).

    The proposal picks one of the N particles and one of the V-N empty sites
    uniformly; acceptance uses the quantised thresholds T (probability
    T/2^32, or 1 for 0xFFFFFFFF).  Returns (states as bitmasks, energies,
    dense float64 matrix P[x, y])."""
    V = chain.volume(d, L)
    states = []
    for combo in itertools.combinations(range(V), N):
        m = 0
        for s in combo:
            m |= 1 << s
        states.append(m)
    index = {m: i for i, m in enumerate(states)}
    energies = np.array([chain.energy_mask(d, L, m) for m in states], dtype=np.int64)
    n = len(states)
    P = np.zeros((n, n))
    prop = 1.0 / (N * (V - N))
    width = 4 * d + 1
    for i, m in enumerate(states):
        occ_sites = [s for s in range(V) if (m >> s) & 1]
        empty_sites = [s for s in range(V) if not (m >> s) & 1]
        e = int(energies[i])
        for a in occ_sites:
            for b in empty_sites:
                de = chain.delta_e_mask(d, L, m, a, b)
                t = int(T[e - e_lo, de + 2 * d]) if 0 <= de + 2 * d < width else 0
                acc = 1.0 if t == 0xFFFFFFFF else t / 4294967296.0
                if acc > 0:
                    y = (m & ~(1 << a)) | (1 << b)
                    P[i, index[y]] += prop * acc
        P[i, i] += 1.0 - P[i].sum()
    return states, energies, P


def reweight_mean_energy(lnW, H, e_lo, beta):
    """<E>_beta from a multicanonical histogram (Sec. 3: reweighting to the
    canonical ensemble): P_beta(E) ~ H(E) exp(-beta E - lnW(E))."""
    num = 0.0
    den = 0.0
    logs = []
    for b in range(len(H)):
        if H[b] > 0:
            e = e_lo + b
            logs.append((e, math.log(float(H[b])) - beta * e - lnW[b]))
    mx = max(v for _, v in logs)
    for e, v in logs:
        w = math.exp(v - mx)
        num += w * e
        den += w
    return num / den


def reweight_moments(lnW, H, e_lo, beta):
    """(<E>_beta, <E^2>_beta) from a multicanonical histogram sampled with
    weights lnW (Sec. 3: the data are reweighted to the temperatures of
    interest): P_beta(E) ~ H(E) exp(-beta E - lnW(E))."""
    logs = []
    for b in range(len(H)):
        if H[b] > 0:
            e = e_lo + b
            logs.append((e, math.log(float(H[b])) - beta * e - lnW[b]))
    mx = max(v for _, v in logs)
    m0 = m1 = m2 = 0.0
    for e, v in logs:
        w = math.exp(v - mx)
        m0 += w
        m1 += w * e
        m2 += w * e * e
    return m1 / m0, m2 / m0


def reweight_observable(lnW, H, e_lo, beta, obs):
    """Canonical mean at beta of a microcanonical observable obs[b] (NaN where
    unmeasured) from a multicanonical histogram (Sec. 3): weights
    H(E) exp(-beta E - lnW(E)) over bins with H > 0 and finite obs."""
    logs = []
    for b in range(len(H)):
        if H[b] > 0 and math.isfinite(obs[b]):
            logs.append((b, math.log(float(H[b])) - beta * (e_lo + b) - lnW[b]))
    if not logs:
        return float("nan")
    mx = max(v for _, v in logs)
    z = s = 0.0
    for b, v in logs:
        w = math.exp(v - mx)
        z += w
        s += w * obs[b]
    return s / z


def exact_moments(omega: dict, beta: float):
    """(<E>_beta, <E^2>_beta) from an exact density of states (Eq. 1)."""
    mx = max(-beta * e for e in omega)
    z = sum(c * math.exp(-beta * e - mx) for e, c in omega.items())
    m1 = sum(c * e * math.exp(-beta * e - mx) for e, c in omega.items())
    m2 = sum(c * e * e * math.exp(-beta * e - mx) for e, c in omega.items())
    return m1 / z, m2 / z


def exact_mean_energy(omega: dict, beta: float) -> float:
    """<E>_beta from an exact density of states (Eq. 1, canonical)."""
    mx = max(-beta * e for e in omega)
    num = sum(c * e * math.exp(-beta * e - mx) for e, c in omega.items())
    den = sum(c * math.exp(-beta * e - mx) for e, c in omega.items())
    return num / den


def ising_constant(d, L, N, J=1.0):
    """c(N) of Eq. 5: H_gas = H_Ising / 4 + c(N) with s_i = 2 n_i - 1.

    Summing s_i s_j = 4 n_i n_j - 2 n_i - 2 n_j + 1 over the dV bonds, each
    site lying on 2d bonds, gives sum s_i s_j = 4 sum n_i n_j - 4dN + dV,
    hence c(N) = J d (V/4 - N)."""
    V = chain.volume(d, L)
    return J * d * (V / 4.0 - N)


def ising_energy_of_occ(d, L, occ):
    """-J sum_<ij> s_i s_j with s = 2n - 1, counted directly from the spins."""
    V = chain.volume(d, L)
    s = 2 * np.asarray(occ, dtype=np.int64) - 1
    tot = 0
    for site in range(V):
        nb = chain.neighbours(d, L, site)
        for k in range(d):
            tot += s[site] * s[nb[2 * k + 1]]
    return -tot
