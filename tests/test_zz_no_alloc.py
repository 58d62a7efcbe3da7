"""The allocation-free entry point against the regular one.

mucal_run_walkers_noalloc serves callers that cannot allocate device memory
(for example code that must live inside another framework's memory pool or
within a fixed device-memory budget): it runs one iteration of the walker
update and histogram sum on buffers the caller owns, with its scratch in a
fixed array inside the library.  Here the regular context is the reference:
both start from the same walker states and thresholds, and two calls in a
row must give bit-identical histograms and walker energies (integer results,
so the tolerance of the other parity tests is exact equality).  The device
buffers of the allocation-free side are created by this test with torch; the
entry point itself allocates nothing.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

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


def _device_state(mc, info):
    """Copy every walker's state of a regular context into torch device tensors
    laid out as the allocation-free call expects."""
    import torch
    W, V = info["n_walkers"], info["V"]
    words = (V + 31) // 32
    bits = np.zeros((W, words), dtype=np.uint32)
    S = np.zeros((W, V), dtype=np.uint16 if V <= 65536 else np.uint32)
    E = np.zeros(W, dtype=np.int32)
    for w in range(W):
        occ, s, e = mc.walker_state(0, w)
        padded = np.zeros(words * 32, dtype=np.uint8)
        padded[:V] = occ
        bits[w] = np.packbits(padded, bitorder="little").view("<u4")
        S[w] = s
        E[w] = e
    dev = torch.device("cuda")
    t_bits = torch.from_numpy(bits.view(np.int32)).to(dev)
    t_S = torch.from_numpy(S.view(np.int16 if S.dtype == np.uint16 else np.int32)).to(dev)
    t_E = torch.from_numpy(E).to(dev)
    return t_bits, t_S, t_E


@pytest.mark.parametrize("desc,sweeps", [
    ((2, 32, 102, 300, 0, 0, 11), 40),
    ((3, 12, 173, 97, 0, 0, 5000), 15),
])
def test_noalloc_matches_regular_entry_point_twice(desc, sweeps):
    import torch
    d, L, N, W, lo, hi, seed = desc
    with m.Mucal([desc]) as mc:
        info = mc.info[0]
        lnW = workloads.random_log_weights(info["n_bins"], 21, scale=0.1)
        mc.set_weights(0, lnW)
        thr = mc.thresholds(0)
        t_bits, t_S, t_E = _device_state(mc, info)
        t_thr = torch.from_numpy(thr.view(np.int32).copy()).cuda()
        t_H = torch.zeros(info["n_bins"], dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        for it in range(2):
            mc.run_iteration(sweeps, it)
            H_ref = mc.histogram(0)
            m.mucal_run_walkers_noalloc(desc, sweeps, it, t_bits.data_ptr(), t_S.data_ptr(),
                                        t_E.data_ptr(), t_thr.data_ptr(), t_H.data_ptr(),
                                        stream.cuda_stream)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(t_H.cpu().numpy(), H_ref)
            assert int(H_ref.sum()) == W * sweeps * N
            E_ref = np.array([mc.walker_state(0, w)[2] for w in range(W)], dtype=np.int32)
            np.testing.assert_array_equal(t_E.cpu().numpy(), E_ref)
