"""The two-stage iteration driver (iterate_staged) on the GPU.

From lnW = 0 the first stage must sample the whole range of a small lattice
and the second stage reach a flat histogram; started from the exact weights
1/Omega of an enumerated lattice, the relaxation replaces the first stage
and the first measured histogram is already flat.  Tunnelling events are
counted in stage 2 (the Sec. 4 criterion)."""
import numpy as np
import pytest

from oracle import chain
from paper_1401_4076_gb300 import mucal as m

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


def test_staged_from_zero_samples_range_and_flattens():
    from paper_1401_4076_gb300.iterate import iterate_staged
    r = iterate_staged((2, 16, 32, 256, 0, 0, 5), range_sweeps=100, sweeps=400, discard=100,
                       max_iter=150)
    assert r.converged, r.flatness[-10:]
    assert r.range_iterations >= 5
    # the compact ground state of 32 particles on 16 x 16: 2N - ceil(2 sqrt(N)) = 52 bonds
    assert r.span[0] <= -50 and r.span[1] == 0
    assert r.tunnel_events > 0


def test_staged_from_exact_weights_is_flat_at_once():
    from paper_1401_4076_gb300.iterate import iterate_staged
    om = chain.enumerate_omega(2, 4, 8)
    lnW = np.array([-np.log(om[e]) if e in om else 0.0 for e in range(-16, 1)])
    r = iterate_staged((2, 4, 8, 64, 0, 0, 9), lnW0=lnW, sweeps=2000, discard=200, max_iter=20)
    assert r.converged
    assert r.iterations - r.range_iterations <= 2
    assert np.isnan(r.flatness[:r.range_iterations]).all()
