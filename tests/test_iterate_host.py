"""Host logic of the two-stage iteration driver (no GPU): a scripted stand-in
for the library context drives `iterate_staged` through stage 1 (until the
sampled range is stable) and stage 2 (until the flatness goal), and the
command line's progress lines."""
import json

import numpy as np
import pytest

from paper_1401_4076_gb300 import iterate


class FakeContext:
    """Histograms whose visited range grows for two iterations and then stays,
    and stage-2 flatness values from a script."""

    def __init__(self, systems, cuda_stream=None):
        d, L, N, W, lo, hi, seed = systems[0]
        self.nb = 11
        self.info = [{"e_lo": -10, "n_bins": self.nb}]
        self.it = 0
        self.runs = []
        self.lnW = np.zeros(self.nb)
        self.flat_script = [0.1, 0.3, 0.6, 0.9]
        self.tunnel = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def set_launch(self, **kw):
        pass

    def set_weights(self, s, w):
        self.lnW = np.asarray(w, dtype=float).copy()

    def weights(self, s):
        return self.lnW.copy()

    def set_target_window(self, s, lo, hi):
        pass

    def set_tunnel_window(self, s, lo, hi):
        self.tunnel_window = (lo, hi)

    def run_iteration(self, sweeps, it):
        self.runs.append((sweeps, it))
        self.it += 1
        self.tunnel += 2

    def histogram(self, s):
        H = np.zeros(self.nb, dtype=np.int64)
        lo, hi = {1: (4, 6), 2: (3, 7)}.get(self.it, (2, 8))
        H[lo:hi + 1] = 5
        return H

    def update_weights(self, s, scheme):
        f = self.flat_script.pop(0) if self.stage2 else 0.0
        return self.lnW, f

    def tunnel_counts(self, s):
        return self.tunnel, None, None

    stage2 = False


@pytest.fixture
def fake(monkeypatch):
    made = []

    class Ctx(FakeContext):
        def __init__(self, *a, **k):
            super().__init__(*a, **k)
            made.append(self)

        def set_tunnel_window(self, s, lo, hi):
            super().set_tunnel_window(s, lo, hi)
            self.stage2 = True        # stage 2 starts by setting the tunnelling window

    monkeypatch.setattr(iterate.m, "Mucal", Ctx)
    return made


def test_staged_stages_and_progress(fake):
    seen = []
    r = iterate.iterate_staged((2, 8, 5, 4, 0, 0, 0), range_sweeps=10, sweeps=40, discard=5,
                               max_iter=50, stable=3, progress=seen.append)
    ctx = fake[0]
    # stage 1: ranges (4,6), (3,7), then (2,8) three more times until stable for 3
    assert r.range_iterations == 6
    assert r.span == (-10 + 2, -10 + 8)
    assert ctx.tunnel_window == (-8, -2)
    # stage 2: flatness 0.1, 0.3, 0.6 -> converged at the third
    assert r.converged and r.iterations == 6 + 3
    assert [p["stage2_iteration"] for p in seen] == [1, 2, 3]
    assert [p["flatness"] for p in seen] == [0.1, 0.3, 0.6]
    assert [p["iteration"] for p in seen] == [7, 8, 9]
    # each stage-2 iteration is a discarded run and a measured run
    assert r.sweeps == 6 * 10 + 3 * (5 + 40)
    assert [sw for sw, _ in ctx.runs[6:]] == [5, 40, 5, 40, 5, 40]
    its = [it for _, it in ctx.runs]
    assert its == list(range(len(its)))        # iteration numbers never repeat


def test_staged_without_progress_is_unchanged(fake):
    r = iterate.iterate_staged((2, 8, 5, 4, 0, 0, 0), range_sweeps=10, sweeps=40, discard=5,
                               max_iter=50, stable=3)
    assert r.converged and r.iterations == 9


def test_staged_cap_counts_both_stages(fake):
    r = iterate.iterate_staged((2, 8, 5, 4, 0, 0, 0), range_sweeps=10, sweeps=40, discard=0,
                               max_iter=8, stable=3, goal=0.95)
    assert not r.converged and r.iterations == 8 and r.range_iterations == 6


def test_cli_progress_lines(fake, capsys):
    iterate.main(["--system", "2:8:5:4", "--staged", "--range-sweeps", "10", "--sweeps", "40",
                  "--discard", "5", "--max-iter", "50", "--scheme", "simple", "--extrapolate",
                  "--progress", "2"])
    lines = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    prog = [x for x in lines if "stage2_iteration" in x]
    assert [x["stage2_iteration"] for x in prog] == [2]
    run = [x for x in lines if "stages" in x][0]
    # the command line keeps stable = 5: ranges (4,6), (3,7), then (2,8) six times
    assert run["range_iterations"] == 8
    assert run["converged"] and run["iterations"] == 8 + 3 and lines[-1]["summary"]


class FakeMulti:
    """Several systems in one context; system i reports the flatness values
    of its script, and histograms whose mean energy bin is scripted too."""

    scripts = {}
    means = {}

    def __init__(self, systems, cuda_stream=None):
        self.systems = systems
        self.nb = 9
        self.it = [0] * len(systems)
        self.runs = []
        self.updates = [0] * len(systems)
        self.w = [np.zeros(self.nb) for _ in systems]
        FakeMulti.last = self

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def set_launch(self, **kw):
        pass

    def set_weights(self, i, w):
        self.w[i] = np.asarray(w, float).copy()

    def weights(self, i):
        return self.w[i].copy()

    def set_target_window(self, i, lo, hi):
        pass

    def run_iteration(self, sweeps, it):
        self.runs.append((sweeps, it))

    def histogram(self, i):
        k = len(self.runs)
        c = FakeMulti.means.get(i, lambda k: 4)(k)
        H = np.zeros(self.nb, dtype=np.int64)
        H[c] = 10
        return H

    def update_weights(self, i, scheme):
        s = FakeMulti.scripts[i]
        f = s[min(self.updates[i], len(s) - 1)]
        self.updates[i] += 1
        return self.w[i], f


@pytest.fixture
def multi(monkeypatch):
    monkeypatch.setattr(iterate.m, "Mucal", FakeMulti)
    FakeMulti.scripts, FakeMulti.means = {}, {}
    return FakeMulti


def test_iterate_to_flat_per_system_convergence(multi):
    multi.scripts = {0: [0.1, 0.6], 1: [0.1, 0.2, 0.3, 0.7]}
    sysd = [(2, 8, 5, 4, 0, 0, 0), (2, 8, 6, 4, 0, 0, 4)]
    res = iterate.iterate_to_flat(sysd, sweeps=10, max_iter=20, scheme=0, final_sweeps=30)
    assert [r.converged for r in res] == [True, True]
    assert [r.iterations for r in res] == [2, 4]
    assert res[0].flatness == [0.1, 0.6] and res[1].flatness == [0.1, 0.2, 0.3, 0.7]
    # a converged system keeps running with frozen weights (no more updates)
    assert multi.last.updates == [2, 4]
    # one launch per iteration for all systems, then the final run
    assert [sw for sw, _ in multi.last.runs] == [10, 10, 10, 10, 30]
    assert res[0].attempts == 2 * 10 * 5 * 4 and res[1].attempts == 4 * 10 * 6 * 4


def test_iterate_to_flat_sweeps_double_on_stalls(multi):
    multi.scripts = {0: [0.1] * 40}
    res = iterate.iterate_to_flat([(2, 8, 5, 4, 0, 0, 0)], sweeps=10, max_iter=12, scheme=0,
                                  sweeps_growth=4, stall=3)
    sw = res[0].extra["sweeps"]
    # best improves once (first value), then 3 stalled iterations double the sweeps,
    # twice, up to 4 times the start
    assert sw[0] == 10 and max(sw) == 40 and sorted(set(sw)) == [10, 20, 40]
    assert not res[0].converged and res[0].iterations == 12


def test_iterate_to_flat_relaxation_ends_when_the_mean_settles(multi):
    multi.scripts = {0: [0.9]}
    # mean energy bin 6, 5, 4, 4, ...: settles at the fourth iteration
    multi.means = {0: lambda k: max(4, 7 - k)}
    res = iterate.iterate_to_flat([(2, 8, 5, 4, 0, 0, 0)], sweeps=10, max_iter=20, scheme=0,
                                  lnW0=[np.linspace(0, -1, 9)], relax_iters=10, relax_tol=0.05)
    fl = res[0].flatness
    n_relax = sum(1 for x in fl if x != x)
    assert n_relax == 4 and fl[-1] == 0.9 and res[0].converged
    assert res[0].iterations == n_relax + 1
