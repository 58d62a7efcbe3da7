"""The tcgen05 passes of the seeding network (the default) against the
mma.sync ones and the float64 oracle (same bf16-rounded parameters).  The
two GPU paths differ only in the order of their fp32 sums."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


@pytest.mark.parametrize("B", [1, 127, 128, 129, 1000, 4097])
def test_tcgen05_forward_matches_mma_and_oracle(B):
    params = workloads.mlp_initial_params(5)
    X, t = workloads.mlp_test_batch(max(B, 256), 6)
    with m.Mlp(params) as net:
        net.train(X, t, steps=200, lr=2e-3)       # weights away from their start
        Xb = X[:B]
        y_tc = net.forward_tcgen05(Xb)
        net.use_tcgen05(False)
        y_mma = net.forward(Xb)
        q = net.params(rounded=True)
    po = {k: np.asarray(v, dtype=np.float64) for k, v in m.mlp_unflatten(q).items()}
    yo, _ = omlp.forward(po, Xb.astype(np.float64))
    scale = max(1.0, float(np.abs(yo).max()))
    assert np.abs(y_tc - y_mma).max() <= 1e-5 * scale
    assert np.abs(y_tc - yo).max() <= 1e-2 * scale


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12))


@pytest.mark.parametrize("B", [50, 128, 1000, 3001])
def test_tcgen05_gradients_match_mma_and_oracle(B):
    params = workloads.mlp_initial_params(7)
    X, t = workloads.mlp_test_batch(B, 8)
    with m.Mlp(params) as net:
        net.use_tcgen05(False)
        loss_m, g_m = net.gradients(X, t)
        net.use_tcgen05(True)
        loss_t, g_t = net.gradients(X, t)
        q = net.params(rounded=True)
    po = {k: np.asarray(v, dtype=np.float64) for k, v in m.mlp_unflatten(q).items()}
    lo = omlp.loss(po, X.astype(np.float64), t.astype(np.float64))
    go = omlp.backward(po, X.astype(np.float64), t.astype(np.float64))
    assert loss_t == pytest.approx(loss_m, rel=1e-4)
    assert abs(loss_t - lo) <= 1e-2 * max(lo, 1e-6)
    gt, gm = m.mlp_unflatten(g_t), m.mlp_unflatten(g_m)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a = np.asarray(gt[name], dtype=np.float64).reshape(-1)
        b = np.asarray(gm[name], dtype=np.float64).reshape(-1)
        o = go[name].reshape(-1)
        assert _rel(a, b) <= 1e-2, (name, _rel(a, b))
        assert _rel(a, o) <= 2e-2, (name, _rel(a, o))
        cos = float(a @ o / max(np.linalg.norm(a) * np.linalg.norm(o), 1e-30))
        assert cos >= 0.999, (name, cos)


def test_tcgen05_training_lowers_the_loss_like_mma():
    params = workloads.mlp_initial_params(9)
    X, t = workloads.mlp_test_batch(2000, 10)
    losses = {}
    for tc in (False, True):
        with m.Mlp(params) as net:
            net.use_tcgen05(tc)
            first, _ = net.gradients(X, t)
            last = net.train(X, t, steps=300, lr=2e-3)
            losses[tc] = (first, last)
    for tc, (first, last) in losses.items():
        assert last < 0.5 * first, (tc, first, last)
    assert losses[True][1] == pytest.approx(losses[False][1], rel=0.2)


@pytest.mark.parametrize("B", [300, 8192])
def test_tcgen05_training_is_deterministic(B):
    """Each CTA writes its gradient row and the rows are summed in CTA order,
    so two trainings from the same parameters on the same rows give the same
    parameters to the bit (and so the same seeded weights)."""
    params = workloads.mlp_initial_params(11)
    X, t = workloads.mlp_test_batch(B, 12)
    out = []
    for _ in range(2):
        with m.Mlp(params) as net:
            loss = net.train(X, t, steps=300, lr=2e-3)
            g_loss, g = net.gradients(X, t)
            out.append((loss, net.params(), g_loss, g))
    (l0, p0, gl0, g0), (l1, p1, gl1, g1) = out
    assert l0 == l1 and gl0 == gl1
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(g0, g1)
