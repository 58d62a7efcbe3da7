"""Pin of the oracle's tunnelling count (Sec. 4: convergence after a number
of travels between the maximal and the minimal energy).

The oracle counts events inside its chain, checking every energy the walker
takes.  Here the same chains are advanced one attempt per call, the energy
trace is recorded, and the events are counted a second way: label every
energy at or below e_min 'L' and at or above e_max 'H', drop the rest,
collapse repeated labels; the events are the collapsed length minus one.
"""
import numpy as np

from oracle import chain


def _collapse_count(trace, e_min, e_max):
    labels = ["L" if e <= e_min else "H" for e in trace if e <= e_min or e >= e_max]
    runs = [x for i, x in enumerate(labels) if i == 0 or labels[i - 1] != x]
    return max(len(runs) - 1, 0), (runs[-1] if runs else None)


def test_tunnel_count_matches_trace_collapse():
    d, L, N, W = 2, 4, 5, 24
    e_lo, e_hi = -d * N, 0
    # multicanonical weights 1/Omega from the enumeration: the walkers roam
    omega = chain.enumerate_omega(d, L, N)
    lnW = np.array([-np.log(omega[e]) if e in omega else 0.0 for e in range(e_lo, e_hi + 1)])
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    S, occ, E = chain.init_walkers(d, L, N, W, 300)
    e_min, e_max = -5, 0           # the lowest and highest energies of 4x4, N = 5
    tstate = np.zeros(W, np.uint8)
    tcount = np.zeros(W, np.int64)
    traces = [[int(e)] for e in E]
    for it in range(3000):
        chain.run_walkers_tunnel(d, L, N, 300, it, 1, e_lo, e_hi, T, S, occ, E, e_min, e_max,
                                 tstate, tcount)
        for w in range(W):
            traces[w].append(int(E[w]))
    total = 0
    for w in range(W):
        n, last = _collapse_count(traces[w], e_min, e_max)
        assert tcount[w] == n, (w, tcount[w], n)
        assert tstate[w] == {None: 0, "L": 1, "H": 2}[last]
        total += n
    assert total > 3 * W          # the walkers really travel


def test_tunnel_bookkeeping_does_not_change_the_chain():
    d, L, N, W = 2, 6, 9, 8
    e_lo, e_hi = -d * N, 0
    T = chain.thresholds(d, e_lo, e_hi, np.linspace(0, 6, e_hi - e_lo + 1)[::-1].copy())
    S1, occ1, E1 = chain.init_walkers(d, L, N, W, 5)
    S2, occ2, E2 = S1.copy(), occ1.copy(), E1.copy()
    h1, _ = chain.run_walkers(d, L, N, 5, 3, 500, e_lo, e_hi, T, S1, occ1, E1)
    h2 = chain.run_walkers_tunnel(d, L, N, 5, 3, 500, e_lo, e_hi, T, S2, occ2, E2, -10, -2,
                                  np.zeros(W, np.uint8), np.zeros(W, np.int64))
    np.testing.assert_array_equal(h1, h2)
    np.testing.assert_array_equal(S1, S2)
    np.testing.assert_array_equal(E1, E2)
