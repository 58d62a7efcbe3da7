"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake (a flipped sign,
a dropped exclusion, a wrong constant, a double count, a wrong rounding, a
half-followed bond, an inverted exchange),
builds it with gcc into a temporary directory and runs the pin that should
catch it against the mutant.  The pin must fail on every mutant and pass on
the unmodified oracle.  Nothing here touches a GPU.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import build as obuild

SRC = os.path.join(os.path.dirname(obuild.__file__), "mucal_oracle.c")

MUTATIONS = {
    "dE sign flipped": ("return n_a - n_b;", "return n_b - n_a;"),
    "a counted as its own neighbour": ("if (nb[k] != a) n_b += occ[nb[k]];", "n_b += occ[nb[k]];"),
    "Philox key increment wrong": ("k0 += ORC_PHILOX_W0;", "k0 += ORC_PHILOX_W0 + 2u;"),
    "threshold rounded up": ("double x = floor(ldexp(exp(delta), 32));",
                             "double x = ceil(ldexp(exp(delta), 32)) + 4096.0;"),
    "bonds counted twice": ("if (occ[nb[2 * k + 1]]) ++pairs;", "if (occ[nb[2 * k + 1]]) pairs += 2;"),
    "cluster search follows +1 bonds only": ("int64_t t = nb[k];", "int64_t t = nb[k | 1];"),
    "exchange exponent sign flipped": ("double x = (beta[k] - beta[k + 1]) * (double)(E[ia] - E[ib]);",
                                       "double x = (beta[k + 1] - beta[k]) * (double)(E[ia] - E[ib]);"),
}


def _build(tmp_path, name, mutation):
    src = open(SRC).read()
    if mutation is not None:
        old, new = mutation
        assert src.count(old) == 1, name
        src = src.replace(old, new)
    c = tmp_path / (name.replace(" ", "_") + ".c")
    so = tmp_path / (name.replace(" ", "_") + ".so")
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so),
                    str(c), "-lm"], check=True)
    return obuild._bind(ctypes.CDLL(str(so)))


def _p(a):
    return a.ctypes.data


# ---- pins, written against a given compiled oracle -------------------------

def pin_detailed_balance(lib):
    """3x3, N=4, random weights: pi P = pi (exact transition matrix)."""
    import itertools
    d, L, N, V = 2, 3, 4, 9
    rng = np.random.default_rng(4)
    lnW = rng.normal(scale=1.5, size=d * N + 1)
    T = np.zeros((d * N + 1, 4 * d + 1), dtype=np.uint32)
    lib.orc_thresholds(d, -d * N, 0, _p(lnW), _p(T))
    states = []
    for combo in itertools.combinations(range(V), N):
        states.append(sum(1 << s for s in combo))
    index = {s: i for i, s in enumerate(states)}
    en = np.array([lib.orc_energy_mask(d, L, np.uint64(s)) for s in states])
    P = np.zeros((len(states), len(states)))
    for i, s in enumerate(states):
        occ = [v for v in range(V) if (s >> v) & 1]
        emp = [v for v in range(V) if not (s >> v) & 1]
        for a in occ:
            for b in emp:
                de = lib.orc_delta_e_mask(d, L, np.uint64(s), a, b)
                if not -2 * d <= de <= 2 * d:
                    return False
                t = int(T[en[i] + d * N, de + 2 * d])
                acc = 1.0 if t == 0xFFFFFFFF else t / 2.0 ** 32
                y = (s & ~(1 << a)) | (1 << b)
                P[i, index[y]] += acc / (N * (V - N))
        P[i, i] += 1.0 - P[i].sum()
    pi = np.exp(lnW[en + d * N])
    pi /= pi.sum()
    return bool(np.abs(pi @ P - pi).max() < 1e-9)


def pin_energy_roll(lib):
    rng = np.random.default_rng(1)
    for d, L, N in ((2, 6, 12), (3, 4, 20)):
        V = L ** d
        for _ in range(10):
            occ = np.zeros(V, dtype=np.uint8)
            occ[rng.choice(V, N, replace=False)] = 1
            g = occ.astype(np.int64).reshape((L,) * d)
            ref = -int(sum((g * np.roll(g, 1, axis=ax)).sum() for ax in range(d)))
            if lib.orc_energy(d, L, _p(occ)) != ref:
                return False
    return True


def pin_thresholds_bound(lib):
    rng = np.random.default_rng(3)
    d, nb = 2, 41
    lnW = rng.normal(scale=3.0, size=nb)
    T = np.zeros((nb, 4 * d + 1), dtype=np.uint32)
    lib.orc_thresholds(d, -40, 0, _p(lnW), _p(T))
    for b in range(nb):
        for j, de in enumerate(range(-2 * d, 2 * d + 1)):
            if not 0 <= b + de < nb:
                continue
            p = min(1.0, math.exp(lnW[b + de] - lnW[b]))
            if T[b, j] != 0xFFFFFFFF and not (p - 2.0 ** -31 <= int(T[b, j]) / 2.0 ** 32 <= p):
                return False
    return True


def pin_largest_cluster(lib):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(11)
    for d, L in ((2, 6), (3, 4)):
        V = L ** d
        g = nx.grid_graph(dim=[L] * d, periodic=True)
        for _ in range(20):
            occ = (rng.random(V) < 0.45).astype(np.uint8)
            keep = [t for t in g.nodes if occ[sum(int(t[k]) * L ** k for k in range(d))]]
            ref = max((len(c) for c in nx.connected_components(g.subgraph(keep))), default=0)
            if lib.orc_largest_cluster(d, L, _p(occ)) != ref:
                return False
    return True


def pin_tempering_marginals(lib):
    """4x4, N = 5, ladder of 4 temperatures, one sweep between exchanges:
    each temperature's energy distribution against the enumeration."""
    d, L, N, W, V = 2, 4, 5, 256, 16
    betas = np.array([0.2, 0.9, 1.8, 3.0])
    K = len(betas)
    seeds = np.array([1000 * (k + 1) for k in range(K)], dtype=np.uint64)
    e_lo, nb = -d * N, d * N + 1
    S = np.zeros((K, W, V), np.int32)
    occ = np.zeros((K, W, V), np.uint8)
    E = np.zeros((K, W), np.int64)
    for k in range(K):
        lib.orc_init_walkers(d, L, N, W, np.uint64(seeds[k]), _p(S[k]), _p(occ[k]), _p(E[k]))
    T = np.zeros((K, nb, 4 * d + 1), np.uint32)
    for k in range(K):
        lnW = -betas[k] * np.arange(e_lo, 1, dtype=np.float64)
        lib.orc_thresholds(d, e_lo, 0, _p(lnW), _p(T[k]))
    om = np.zeros(nb, np.int64)
    lib.orc_enumerate(d, L, N, _p(om))
    hist = np.zeros((K, nb))
    h = np.zeros((W, nb), np.int64)
    a = np.zeros(W, np.int64)
    acc = np.zeros(K - 1, np.int64)
    for r in range(1500):
        for k in range(K):
            lib.orc_run_walkers(d, L, N, W, np.uint64(seeds[k]), np.uint32(r), 1, e_lo, 0, _p(T[k]),
                                _p(S[k]), _p(occ[k]), _p(E[k]), _p(h), _p(a))
        lib.orc_replica_exchange(K, W, V, _p(seeds), _p(betas), np.uint32(r), r % 2, _p(S), _p(occ),
                                 _p(E), _p(acc))
        if r >= 100:
            for k in range(K):
                hist[k] += np.bincount(E[k] - e_lo, minlength=nb)
    for k in range(K):
        e = -np.arange(nb)                      # om[j] counts energy -j
        q = om * np.exp(-betas[k] * e - (-betas[k] * e).max())
        q = q / q.sum()
        p = np.zeros(nb)
        p[np.arange(nb)] = hist[k][::-1]        # hist index E - e_lo = nb - 1 - j
        p /= p.sum()
        if 0.5 * np.abs(p - q).sum() >= 0.03:
            return False
    return True


def pin_philox_triton(lib, tmp_path):
    here = os.path.dirname(os.path.abspath(__file__))
    rng = np.random.default_rng(7)
    c = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 2**32, size=(64, 2), dtype=np.uint64).astype(np.uint32)
    np.save(tmp_path / "c.npy", c)
    np.save(tmp_path / "k.npy", k)
    r = subprocess.run(["python", os.path.join(here, "philox_triton_ref.py"), str(tmp_path / "c.npy"),
                        str(tmp_path / "k.npy"), str(tmp_path / "o.npy")], capture_output=True,
                       env=dict(os.environ, TRITON_INTERPRET="1"), timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable")
    ref = np.load(tmp_path / "o.npy")
    out = np.zeros_like(c)
    lib.orc_philox_batch(64, _p(c), _p(k), _p(out))
    return bool(np.array_equal(out, ref))


CASES = [
    ("dE sign flipped", "detailed balance"),
    ("a counted as its own neighbour", "detailed balance"),
    ("Philox key increment wrong", "philox"),
    ("threshold rounded up", "thresholds"),
    ("bonds counted twice", "energy"),
    ("cluster search follows +1 bonds only", "largest cluster"),
    ("exchange exponent sign flipped", "tempering marginals"),
]


def _run_pin(kind, lib, tmp_path):
    if kind == "detailed balance":
        return pin_detailed_balance(lib)
    if kind == "energy":
        return pin_energy_roll(lib)
    if kind == "thresholds":
        return pin_thresholds_bound(lib)
    if kind == "tempering marginals":
        return pin_tempering_marginals(lib)
    if kind == "largest cluster":
        return pin_largest_cluster(lib)
    if kind == "philox":
        pytest.importorskip("triton")
        return pin_philox_triton(lib, tmp_path)
    raise KeyError(kind)


@pytest.mark.parametrize("mutant,pin", CASES)
def test_pin_catches_planted_mistake(tmp_path, mutant, pin):
    assert _run_pin(pin, _build(tmp_path, "clean", None), tmp_path)
    assert not _run_pin(pin, _build(tmp_path, mutant, MUTATIONS[mutant]), tmp_path)


# ---- the Python part of the oracle: the edge continuation of the weights ----

RECURSION_SRC = os.path.join(os.path.dirname(obuild.__file__), "recursion.py")

PY_MUTATIONS = {
    "edge slope sign flipped": ("new[b] = new[first] + slope_lo * (b - first)",
                                "new[b] = new[first] - slope_lo * (b - first)"),
    "edge slope from the wrong member": ("inner_lo = members[kk]", "inner_lo = members[kk - 1]"),
    "upper edge continued flat": ("new[b] = new[last] + slope_hi * (b - last)", "new[b] = new[last]"),
}


def _mutant_recursion(mutation):
    import types
    src = open(RECURSION_SRC).read()
    if mutation is not None:
        old, new = mutation
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    mod = types.ModuleType("recursion_mutant")
    exec(compile(src, "recursion_mutant", "exec"), mod.__dict__)
    return mod


def _edge_pins(mod):
    """The two edge-continuation pins of test_oracle_recursion, on a module."""
    rng = np.random.default_rng(3)
    nb, lo, hi, beta = 60, 10, 45, 0.7
    s_cum = np.zeros(nb, bool)
    s_cum[lo:hi + 1] = True
    E = np.arange(nb) - nb
    lnW = np.where(s_cum, -beta * E, rng.normal(size=nb))
    out = mod.extrapolate_edges(lnW, s_cum)
    shift = out[lo] - lnW[lo]
    ok = (np.allclose(out[:lo] - shift, -beta * E[:lo], atol=1e-9) and
          np.allclose(out[hi + 1:] - shift, -beta * E[hi + 1:], atol=1e-9))
    lnW = np.zeros(12)
    s_cum = np.zeros(12, bool)
    s_cum[[2, 3, 4, 5, 9]] = True
    lnW[[2, 3, 4, 5, 9]] = [7.0, 5.0, 4.0, 3.0, 0.0]
    out1 = mod.extrapolate_edges(lnW, s_cum, k=1)
    expect1 = np.array([11, 9, 7, 5, 4, 3, 0, 0, 0, 0, -0.75, -1.5]) - 11.0
    return ok and np.allclose(out1, expect1, atol=1e-12)


def test_edge_pins_pass_on_the_oracle():
    assert _edge_pins(_mutant_recursion(None))


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_edge_pins_catch_planted_mistakes(name):
    with np.errstate(all="ignore"):          # a mutant may divide by zero
        assert not _edge_pins(_mutant_recursion(PY_MUTATIONS[name])), name
