"""GPU parity of the weight-seeding network against the float64 oracle.

The oracle runs with the bf16-rounded parameters the GPU computes with, so
the remaining differences are the GPU's bf16 activations in the 128x128
contractions and fp32 accumulation: outputs within 1e-2 relative, gradients
with cosine >= 0.999 and relative L2 error <= 2e-2 per tensor.
"""
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


def _oracle_params(vec):
    return {k: np.asarray(v, dtype=np.float64).copy() for k, v in m.mlp_unflatten(vec).items()}


@pytest.mark.parametrize("B", [1, 63, 1000, 4097])
def test_forward_matches_oracle(B):
    params = workloads.mlp_initial_params(1)
    X, _ = workloads.mlp_test_batch(B, 2)
    with m.Mlp(params) as net:
        y = net.forward(X)
        q = net.params(rounded=True)
    yo, _ = omlp.forward(_oracle_params(q), X.astype(np.float64))
    scale = max(1.0, float(np.abs(yo).max()))
    assert np.abs(y - yo).max() <= 1e-2 * scale


@pytest.mark.parametrize("B", [50, 1000, 3000])
def test_gradients_match_oracle(B):
    params = workloads.mlp_initial_params(3)
    X, t = workloads.mlp_test_batch(B, 4)
    with m.Mlp(params) as net:
        loss, g = net.gradients(X, t)
        q = net.params(rounded=True)
    po = _oracle_params(q)
    lo = omlp.loss(po, X.astype(np.float64), t.astype(np.float64))
    go = omlp.backward(po, X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) <= 1e-2 * max(lo, 1e-6)
    gg = m.mlp_unflatten(g)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a = np.asarray(gg[name], dtype=np.float64).reshape(-1)
        b = go[name].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        assert rel <= 2e-2, (name, rel)
        if b.size > 1:
            assert cos >= 0.999, (name, cos)


def test_training_reduces_loss_and_keeps_master_copy():
    params = workloads.mlp_initial_params(5)
    X, t = workloads.mlp_test_batch(2048, 6)
    with m.Mlp(params) as net:
        l0, _ = net.gradients(X, t)
        l1 = net.train(X, t, steps=300, lr=3e-3)
        l2, _ = net.gradients(X, t)
        w = net.params()
        q = net.params(rounded=True)
    assert l2 < 0.2 * l0, (l0, l1, l2)
    assert not np.array_equal(w, params)
    # the rounded copy is the master copy rounded to bf16 (round to nearest even)
    wb = w.view(np.uint32).astype(np.uint64)
    rne = ((wb + 0x7FFF + ((wb >> 16) & 1)) >> 16) << 16
    np.testing.assert_array_equal(q.view(np.uint32), rne.astype(np.uint32))
