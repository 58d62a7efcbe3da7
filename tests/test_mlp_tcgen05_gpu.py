"""The tcgen05 forward pass of the seeding network against the mma.sync one
and the float64 oracle (same bf16-rounded parameters).  The two GPU paths
differ only in the order of their fp32 sums."""
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
        y_mma = net.forward(Xb)
        q = net.params(rounded=True)
    po = {k: np.asarray(v, dtype=np.float64) for k, v in m.mlp_unflatten(q).items()}
    yo, _ = omlp.forward(po, Xb.astype(np.float64))
    scale = max(1.0, float(np.abs(yo).max()))
    assert np.abs(y_tc - y_mma).max() <= 1e-5 * scale
    assert np.abs(y_tc - yo).max() <= 1e-2 * scale
