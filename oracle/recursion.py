"""Weight iteration, flatness and ln Omega in float64 (test infrastructure only).

Energies are held as bins b = E - e_lo of the window [e_lo, e_hi].  Plain
loops in the order the steps are stated; no vectorised shortcuts where a
loop reads closer to the definition.

Readings of what the paper leaves open (each also listed in the design notes):

* Unvisited bins (H = 0) keep their log-weight in the simple iteration; the
  paper states W^{i+1} = W^i / H^i only where H^i > 0 makes sense.
* The recursive scheme is named (Sec. 2) but not written out.  It is read as
  the accumulated-statistics recursion on the ratios R(E) = W(E)/W(E_prev)
  of consecutive energies E_prev < E of the cumulative visited set S_cum:
  g = H(E_prev) H(E) / (H(E_prev) + H(E)) (0 if either is 0),
  p(E) <- p(E) + g, kappa = g / p(E),
  ln R(E) <- ln R(E) + kappa (ln H(E_prev) - ln H(E)).
  The weights are rebuilt from the top member of S_cum downwards.  Bins
  outside S_cum keep their log-weight offset to the nearest member above
  them (below, if there is none above).
* Optional edge continuation (a reading of the recursion's boundary
  treatment, which the paper leaves open): after an update, bins below the
  lowest member of S_cum and above the highest take lnW continued linearly
  with the slope between the edge member and the k-th member counted inwards
  from it (k = 8, or the last member if S_cum is smaller), i.e. canonical
  weights at the microcanonical inverse temperature of the sampled edge,
  instead of the flat continuation of the plain schemes.
* After every update lnW is shifted so that its maximum over the window is 0.
* Flatness: min over S_cum of H / max of H, or -1 while either end of the
  target window has not been visited (the flatness goal min/max >= 0.5).
"""
from __future__ import annotations

import math

import numpy as np


def normalise(lnW: np.ndarray) -> np.ndarray:
    """Shift so that max lnW = 0 (acceptance ratios are unchanged)."""
    out = np.array(lnW, dtype=np.float64, copy=True)
    return out - out.max()


def simple_update(lnW: np.ndarray, H: np.ndarray) -> np.ndarray:
    """W^{i+1}(E) = W^i(E) / H^i(E) (Sec. 2) in logs, for bins with H > 0."""
    new = np.array(lnW, dtype=np.float64, copy=True)
    for b in range(len(new)):
        if H[b] > 0:
            new[b] = lnW[b] - math.log(float(H[b]))
    return normalise(new)


def recursive_update(lnW: np.ndarray, H: np.ndarray, s_cum: np.ndarray, phat: np.ndarray):
    """Accumulated-statistics recursion (reading of the scheme cited in Sec. 2).

    ``s_cum`` (bool) and ``phat`` (float64) are the recursion memory; new
    copies are returned as (lnW_new, s_cum_new, phat_new).
    """
    n = len(lnW)
    s_cum = np.array(s_cum, dtype=bool, copy=True)
    phat = np.array(phat, dtype=np.float64, copy=True)
    for b in range(n):
        if H[b] > 0:
            s_cum[b] = True
    members = [b for b in range(n) if s_cum[b]]
    new = np.array(lnW, dtype=np.float64, copy=True)
    if not members:
        return normalise(new), s_cum, phat
    top = members[-1]
    new[top] = lnW[top]
    for j in range(len(members) - 1, 0, -1):
        hi = members[j]
        lo = members[j - 1]
        ln_r = lnW[hi] - lnW[lo]
        h_lo = float(H[lo])
        h_hi = float(H[hi])
        if h_lo > 0 and h_hi > 0:
            g = h_lo * h_hi / (h_lo + h_hi)
        else:
            g = 0.0
        phat[hi] = phat[hi] + g
        if g > 0:
            kappa = g / phat[hi]
            ln_r = ln_r + kappa * (math.log(h_lo) - math.log(h_hi))
        new[lo] = new[hi] - ln_r
    for b in range(n):
        if s_cum[b]:
            continue
        above = [m for m in members if m > b]
        ref = above[0] if above else members[-1]
        new[b] = lnW[b] + (new[ref] - lnW[ref])
    return normalise(new), s_cum, phat


EDGE_MEMBERS = 8


def extrapolate_edges(lnW: np.ndarray, s_cum: np.ndarray, k: int = EDGE_MEMBERS) -> np.ndarray:
    """Continue lnW linearly beyond both ends of the cumulative visited set:
    below its lowest member with the slope from that member to the k-th
    member above it, above its highest member with the slope from the k-th
    member below it.  Bins between members are left as they are.  Returns
    a new array shifted to max 0; unchanged (but shifted) with fewer than two
    members."""
    new = np.array(lnW, dtype=np.float64, copy=True)
    members = [b for b in range(len(new)) if s_cum[b]]
    if len(members) < 2:
        return normalise(new)
    kk = min(k, len(members) - 1)
    first, last = members[0], members[-1]
    inner_lo = members[kk]
    inner_hi = members[len(members) - 1 - kk]
    slope_lo = (new[inner_lo] - new[first]) / (inner_lo - first)
    slope_hi = (new[last] - new[inner_hi]) / (last - inner_hi)
    for b in range(0, first):
        new[b] = new[first] + slope_lo * (b - first)
    for b in range(last + 1, len(new)):
        new[b] = new[last] + slope_hi * (b - last)
    return normalise(new)


def flatness(H: np.ndarray, s_cum: np.ndarray, t_lo_bin: int | None = None,
             t_hi_bin: int | None = None) -> float:
    """min/max of H over S_cum within the target window; -1 if an end is unvisited."""
    members = [b for b in range(len(H)) if s_cum[b]]
    if not members:
        return -1.0
    lo = members[0] if t_lo_bin is None else t_lo_bin
    hi = members[-1] if t_hi_bin is None else t_hi_bin
    if not s_cum[lo] or not s_cum[hi]:
        return -1.0
    vals = [float(H[b]) for b in members if lo <= b <= hi]
    mx = max(vals)
    if mx <= 0:
        return 0.0
    return min(vals) / mx


def ln_omega(lnW: np.ndarray, H: np.ndarray, V: int, N: int) -> np.ndarray:
    """ln Omega(E) = ln H(E) - lnW(E) on bins with H > 0 (W = 1/Omega gives a flat H,
    Sec. 2), shifted so that sum_E Omega(E) = C(V, N).  NaN where H = 0."""
    out = np.full(len(H), np.nan)
    for b in range(len(H)):
        if H[b] > 0:
            out[b] = math.log(float(H[b])) - lnW[b]
    vis = ~np.isnan(out)
    m = out[vis].max()
    lse = m + math.log(sum(math.exp(x - m) for x in out[vis]))
    ln_total = math.lgamma(V + 1) - math.lgamma(N + 1) - math.lgamma(V - N + 1)
    out[vis] += ln_total - lse
    return out


def multi_histogram(H, lnW, max_iter=10000, tol=1e-12):
    """ln Omega from several histograms H_k sampled with weights lnW_k, the
    self-consistent multi-histogram combination: Omega(E) = sum_k H_k(E) /
    sum_k N_k W_k(E) exp(-f_k), exp(f_k) = sum_E Omega(E) W_k(E), f_0 = 0.
    Plain loops; returns (ln Omega shifted to max 0 with NaN where no
    histogram visits, passes)."""
    H = np.asarray(H, dtype=np.float64)
    lnW = np.asarray(lnW, dtype=np.float64)
    K, nb = H.shape
    Nk = H.sum(axis=1)
    num = H.sum(axis=0)
    f = np.zeros(K)
    lo = np.full(nb, np.nan)
    passes = 0
    for passes in range(1, max_iter + 1):
        for b in range(nb):
            if num[b] <= 0:
                continue
            terms = [math.log(Nk[k]) + lnW[k, b] - f[k] for k in range(K) if Nk[k] > 0]
            mx = max(terms)
            lo[b] = math.log(num[b]) - (mx + math.log(sum(math.exp(t - mx) for t in terms)))
        fn = np.zeros(K)
        for k in range(K):
            terms = [lo[b] + lnW[k, b] for b in range(nb) if num[b] > 0]
            mx = max(terms)
            fn[k] = mx + math.log(sum(math.exp(t - mx) for t in terms))
        fn -= fn[0]
        change = np.abs(fn - f).max()
        f = fn
        if change < tol:
            break
    vis = num > 0
    lo[vis] -= lo[vis].max()
    return lo, passes
