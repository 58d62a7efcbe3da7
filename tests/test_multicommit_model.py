"""The decision procedure of the multi-commit rounds, written out in plain
Python, against the serial chain (no GPU).

The walker kernels decide a batch of G consecutive attempts of one chain in
rounds: at the start of a round every undecided lane evaluates its energy
change on the current state and its acceptance at each energy within 2d of
the current one; the round then steps through the lanes in attempt order,
committing the first clean lane that accepts at the energy reached so far and
rejecting the clean lanes before it, until a lane whose evaluation a commit
invalidated (a committed site next to its sites, one of its list slots moved,
or the energy left the evaluated rows) ends the round.  This test restates
that procedure independently of the CUDA source and checks that it reproduces
the serial chain (jump moves of Sec. 2 with the threshold acceptance) attempt
by attempt: every post-attempt energy, and the state after every batch, on
small 2D and 3D lattices including dense ones and lattices of side 3 where
neighbourhoods overlap, with weights that accept almost everything and with
sloped ones."""
import numpy as np
import pytest

from oracle import chain

SAT = 0xFFFFFFFF


def _accepts(T, E, e_lo, n_bins, dE, d, r2):
    row = E - e_lo
    if row < 0 or row >= n_bins:
        return False
    t = int(T[row, dE + 2 * d])
    return t == SAT or r2 < t


def serial_batch(d, L, N, occ, S, E, e_lo, T, attempts):
    """The serial chain over one batch; returns the post-attempt energies."""
    post = []
    nb = T.shape[0]
    for k, m, r2 in attempts:
        a, b = int(S[k]), int(S[N + m])
        dE = chain.delta_e(d, L, occ, a, b)
        if _accepts(T, E, e_lo, nb, dE, d, r2):
            occ[a], occ[b] = 0, 1
            S[k], S[N + m] = b, a
            E += dE
        post.append(E)
    return E, post


def rounds_batch(d, L, N, occ, S, E, e_lo, T, attempts):
    """The multi-commit rounds over one batch; returns the post-attempt
    energies in attempt order, the number of rounds and of commits."""
    G = len(attempts)
    O = 2 * d
    nb = T.shape[0]
    k = [int(x[0]) for x in attempts]
    m = [int(x[1]) for x in attempts]
    r2 = [int(x[2]) for x in attempts]
    a = [int(S[k[j]]) for j in range(G)]        # read at the start of the batch
    b = [int(S[N + m[j]]) for j in range(G)]
    pend = [True] * G
    post = [None] * G
    n_rounds = 0
    n_commits = 0
    while any(pend):
        n_rounds += 1
        dE = [chain.delta_e(d, L, occ, a[j], b[j]) if pend[j] else 0 for j in range(G)]
        acc = [[pend[j] and _accepts(T, E + o, e_lo, nb, dE[j], d, r2[j]) for o in range(-O, O + 1)]
               for j in range(G)]
        nbr = [set(chain.neighbours(d, L, a[j]).tolist()) | set(chain.neighbours(d, L, b[j]).tolist())
               for j in range(G)]
        clean = list(pend)
        off = 0
        while True:
            f = next((j for j in range(G) if pend[j] and clean[j] and acc[j][off + O]), None)
            u = next((j for j in range(G) if pend[j] and not clean[j]), None)
            if u is not None and (f is None or u < f):
                for j in range(u):                  # rejected at the energy reached
                    if pend[j]:
                        pend[j] = False
                        post[j] = E
                break                               # the rest go again next round
            if f is None:
                for j in range(G):                  # nothing accepts: all rejected here
                    if pend[j]:
                        pend[j] = False
                        post[j] = E
                break
            for j in range(f):
                if pend[j]:
                    pend[j] = False
                    post[j] = E
            af, bf = a[f], b[f]
            occ[af], occ[bf] = 0, 1
            S[k[f]], S[N + m[f]] = bf, af
            E += dE[f]
            off += dE[f]
            pend[f] = False
            post[f] = E
            n_commits += 1
            for j in range(f + 1, G):
                if not pend[j]:
                    continue
                if k[j] == k[f]:                    # the moved particle slot now holds bf
                    a[j] = bf
                    clean[j] = False
                if m[j] == m[f]:                    # the used empty-site slot now holds af
                    b[j] = af
                    clean[j] = False
                if af in nbr[j] or bf in nbr[j]:
                    clean[j] = False
                if off > O or off < -O:
                    clean[j] = False
    return E, post, n_rounds, n_commits


CASES = [
    # d, L, N, lanes, weight slope per bin, weight noise, batches, several commits per round?
    (2, 6, 9, 8, 0.0, 0.0, 150, True),     # lnW = 0: every move with dE <= 0 accepted
    (2, 5, 12, 16, -0.8, 0.3, 150, True),  # runs down in energy: long runs of moves
    (2, 3, 4, 8, 0.0, 0.5, 200, None),     # L = 3: neighbourhoods overlap (diagonals do not)
    (2, 8, 40, 32, 0.4, 0.4, 80, True),    # dense, 32 lanes
    (3, 3, 13, 4, 0.0, 0.6, 200, None),    # 3D L = 3: sites overlap almost everywhere
    (3, 4, 20, 16, -0.5, 0.3, 120, True),
    (3, 4, 50, 8, 0.3, 0.5, 120, True),    # dense 3D
    (2, 6, 35, 4, 0.0, 0.0, 150, False),   # one hole: every move uses the same empty-site slot
]


@pytest.mark.parametrize("d,L,N,G,slope,noise,batches,several", CASES)
def test_rounds_reproduce_the_serial_chain(d, L, N, G, slope, noise, batches, several):
    rng = np.random.default_rng(1000 * d + 10 * L + N + G)
    V = L ** d
    e_lo, e_hi = -d * N, 0
    nb = e_hi - e_lo + 1
    lnW = slope * np.arange(nb) + noise * rng.standard_normal(nb)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    S0, occ0, E0 = chain.init_walkers(d, L, N, 1, 77 + N)
    S_s, occ_s, E_s = S0[0].copy(), occ0[0].copy(), int(E0[0])
    S_r, occ_r, E_r = S0[0].copy(), occ0[0].copy(), int(E0[0])
    holes = V - N
    multi = 0
    for _ in range(batches):
        att = [(int(rng.integers(N)), int(rng.integers(holes)), int(rng.integers(1 << 32)))
               for _ in range(G)]
        E_s, post_s = serial_batch(d, L, N, occ_s, S_s, E_s, e_lo, T, att)
        E_r, post_r, n_rounds, n_commits = rounds_batch(d, L, N, occ_r, S_r, E_r, e_lo, T, att)
        assert post_r == post_s
        assert E_r == E_s
        np.testing.assert_array_equal(occ_r, occ_s)
        np.testing.assert_array_equal(S_r, S_s)
        multi += n_rounds < n_commits
    assert E_s == chain.energy(d, L, occ_s)
    if several is not None:
        # several moves committed in one round somewhere in the run, or
        # never where every commit invalidates the later lanes
        assert (multi > 0) == several


@pytest.mark.parametrize("d,L,N,G", [(2, 5, 6, 8), (2, 6, 30, 16), (3, 4, 40, 32), (2, 4, 15, 4)])
def test_moved_slots_found_by_index_or_by_site(d, L, N, G):
    """A commit moves list slots k_f (particle) and N + m_f (empty site).  A
    later lane of the batch holds the entries it read, patched by earlier
    commits; its slot is one the commit moved exactly when its site is the
    committed one (every site sits in exactly one slot), so the kernels may
    find such lanes either way."""
    rng = np.random.default_rng(7 * d + L + N + G)
    V = L ** d
    S0, occ0, E0 = chain.init_walkers(d, L, N, 1, 5 + N)
    S, occ = S0[0].copy(), occ0[0].copy()
    holes = V - N
    checked = 0
    for _ in range(200):
        att = [(int(rng.integers(N)), int(rng.integers(holes))) for _ in range(G)]
        a = [int(S[k]) for k, _ in att]
        b = [int(S[N + m]) for _, m in att]
        for f in range(G):
            if rng.random() < 0.3:
                continue                          # this attempt is rejected
            kf, mf = att[f]
            af, bf = a[f], b[f]
            assert S[kf] == af and S[N + mf] == bf
            occ[af], occ[bf] = 0, 1
            S[kf], S[N + mf] = bf, af
            for j in range(f + 1, G):
                kj, mj = att[j]
                assert (kj == kf) == (a[j] == af)
                assert (mj == mf) == (b[j] == bf)
                checked += 1
                if kj == kf:
                    a[j] = bf
                if mj == mf:
                    b[j] = af
                assert a[j] == S[kj] and b[j] == S[N + mj]
    assert checked > 0
