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
