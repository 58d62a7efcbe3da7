"""Host logic of the learned seeding (no GPU): the seed's weights from the
network's output, and the plain-versus-learned comparison judging both starts
on the same target window."""
import numpy as np

from paper_1401_4076_gb300 import seeding as sd


class FakeNet:
    """Predicts ln Omega / ln C(V, N) as a parabola in the energy feature."""

    def forward(self, X):
        x = X[:, 3].astype(np.float64)
        return (0.5 - 0.4 * x * x).astype(np.float32)


def test_seed_weights_are_minus_ln_omega_shifted_to_zero():
    d, L, N = 2, 16, 40
    e_lo, e_hi = -d * N, 0
    w = sd.seed_weights(FakeNet(), d, L, N, e_lo, e_hi)
    E = np.arange(e_lo, e_hi + 1)
    y = FakeNet().forward(sd.features(d, L, N, E)).astype(np.float64)
    ref = -y * sd.ln_binomial(L ** d, N)
    np.testing.assert_allclose(w, ref - ref.max(), rtol=0, atol=1e-9)
    assert w.max() == 0.0 and len(w) == e_hi - e_lo + 1


def test_features_match_their_definition():
    d, L, N = 3, 10, 150
    E = np.array([-450, -200, 0])
    X = sd.features(d, L, N, E)
    rho = N / L ** d
    np.testing.assert_allclose(X[:, 0], 2 * (d - 2.5))
    np.testing.assert_allclose(X[:, 1], 16.0 / L)
    np.testing.assert_allclose(X[:, 2], 10 * rho - 0.5, rtol=1e-6)
    np.testing.assert_allclose(X[:, 3], 2 * (E / L ** d) / (d * rho) + 1, rtol=1e-6)
    # E = -dN (every particle with all bonds) maps to -1, the gas E = 0 to +1
    assert abs(sd.features(d, L, N, np.array([-d * N]))[0, 3] + 1) < 1e-6


def test_compare_staged_judges_both_on_the_same_target(monkeypatch):
    calls = []

    class R:
        def __init__(self, span):
            self.span = span

    def fake_staged(desc, lnW0=None, seed_range_stage=False, **kw):
        calls.append({"seeded": lnW0 is not None, "target": kw.get("target"),
                      "seed_range_stage": seed_range_stage, "max_iter": kw.get("max_iter")})
        return R((-70, -3))

    monkeypatch.setattr(sd, "iterate_staged", fake_staged)
    desc = (2, 16, 40, 64, 0, 0, 9)
    plain, seeded, seedW = sd.compare_staged(FakeNet(), desc, max_iter=30)
    # no target given: the learned start is judged on the range the plain run sampled
    assert [c["seeded"] for c in calls] == [False, True]
    assert calls[0]["target"] is None and calls[1]["target"] == (-70, -3)
    assert calls[0]["max_iter"] == calls[1]["max_iter"] == 30
    assert len(seedW) == 2 * 40 + 1
    calls.clear()
    sd.compare_staged(FakeNet(), desc, target=(-60, 0), seed_range_stage=True)
    assert [c["target"] for c in calls] == [(-60, 0), (-60, 0)]
    assert [c["seed_range_stage"] for c in calls] == [False, True]
