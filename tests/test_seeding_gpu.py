"""What the trained seeding network gains over the plain start (GPU).

The network is trained on the GPU (the library's own forward and backward
kernels) on ln Omega estimates that converged runs of the method produced on
small lattices (2D L <= 40, 3D L <= 14).  It then seeds a larger lattice,
2D L = 64 at rho = 0.1 with 4096 walkers, over the window [-dN/2, 0].  The
plain method (lnW = 0, recursive scheme) and the seeded start (relaxation,
then the simple scheme) run on the same system and walker seeds; the seeded
run, relaxation iterations included, must reach the flatness goal in fewer
iterations and less wall time (measured over four walker seeds: 21.5 vs 37.5
iterations).
"""
import numpy as np
import pytest

from paper_1401_4076_gb300 import mucal as m
from paper_1401_4076_gb300 import seeding as sd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    m.load_library()


def test_ln_omega_estimate_matches_exact_4x4():
    """The package's ln Omega estimate on a run of the method, 4x4, N = 8:
    within 0.02 of the exact enumeration values."""
    from oracle import chain
    exact = chain.enumerate_omega(2, 4, 8)
    desc = (2, 4, 8, 64, 0, 0, 9)
    r = sd.iterate_to_flat([desc], sweeps=2000, max_iter=40, targets=[(-12, 0)],
                           final_sweeps=200000)[0]
    assert r.converged
    est = sd.ln_omega_estimate(r.lnW, r.H, 16, 8)
    for e, c in exact.items():
        assert abs(est[e + 16] - np.log(c)) < 0.02, (e, est[e + 16], np.log(c))


def test_seeded_start_beats_plain_start():
    small = sd.small_training_systems(0.5, walkers=512)
    res = sd.iterate_to_flat(small, sweeps=100, max_iter=200, final_sweeps=1000)
    assert sum(r.converged for r in res) >= 0.9 * len(res)
    X, t = sd.training_set([r for r in res if r.converged])
    net, loss = sd.train(X, t, steps=20000, lr=1e-3)
    try:
        d, L, rho, W = 2, 64, 0.1, 4096
        N = int(round(rho * L ** d))
        lo, hi = sd.window_fraction(d, N, 0.5)
        plain, seeded, _ = sd.compare_plain_and_seeded(net, (d, L, N, W, lo, hi, 123456), 50, 300)
    finally:
        net.close()
    assert plain.converged and seeded.converged
    assert seeded.iterations < plain.iterations, (seeded.iterations, plain.iterations)
    assert seeded.wall_s < plain.wall_s
