"""The allocation-free entry point against the oracle and the regular one.

mucal_run_walkers_noalloc serves callers that cannot allocate device memory
(code that lives inside another framework's memory pool, or that must stay
within a fixed device-memory budget): it runs one iteration of the walker
update and histogram sum on buffers the caller owns, with its scratch in a
fixed array inside the library.  Two calls in a row must leave every
walker's occupation bitset, site list and energy, and the summed histogram,
exactly where the oracle puts them, and equal to what the regular context
computes from the same start (integer results, so the tolerance of the other
parity tests is exact equality).  Inputs that the device-side check must
catch (an energy outside the window, a list entry that is not a site) are
made on the host; the call must then report MUCAL_ERR_INVALID_ARG and leave
the walker buffers untouched.  The device buffers are created by this test
with torch; the entry point itself allocates nothing.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from oracle import chain
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


def _pack_bits(occ):
    W, V = occ.shape
    words = (V + 31) // 32
    padded = np.zeros((W, words * 32), dtype=np.uint8)
    padded[:, :V] = occ
    return np.packbits(padded, axis=1, bitorder="little").view("<u4").reshape(W, words)


def _to_device(occ, S, E):
    """Walker states laid out as the allocation-free call expects: uint32
    bitsets, uint16 (V <= 65536) or uint32 site lists, int32 energies."""
    import torch
    V = S.shape[1]
    bits = _pack_bits(occ)
    S_t = S.astype(np.uint16 if V <= 65536 else np.uint32)
    dev = torch.device("cuda")
    t_bits = torch.from_numpy(bits.view(np.int32).copy()).to(dev)
    t_S = torch.from_numpy(S_t.view(np.int16 if V <= 65536 else np.int32).copy()).to(dev)
    t_E = torch.from_numpy(E.astype(np.int32)).to(dev)
    return t_bits, t_S, t_E


def _from_device(t_bits, t_S, t_E, V):
    bits = t_bits.cpu().numpy().view(np.uint32)
    S = t_S.cpu().numpy().view(np.uint16 if V <= 65536 else np.uint32).astype(np.int64)
    return bits, S, t_E.cpu().numpy().astype(np.int64)


def _call(desc, sweeps, it, t_bits, t_S, t_E, t_thr, t_H):
    import torch
    stream = torch.cuda.current_stream()
    m.mucal_run_walkers_noalloc(desc, sweeps, it, t_bits.data_ptr(), t_S.data_ptr(),
                                t_E.data_ptr(), t_thr.data_ptr(), t_H.data_ptr(),
                                stream.cuda_stream)


CASES = [
    ((2, 32, 102, 300, 0, 0, 11), 40),        # 2D, uint16 lists, ragged last block
    ((3, 12, 173, 97, 0, 0, 5000), 15),       # 3D
    ((2, 257, 300, 40, 0, 0, 5), 3),          # V = 66049: uint32 lists, bitsets in global memory
]


@pytest.mark.parametrize("desc,sweeps", CASES)
def test_noalloc_matches_oracle_and_regular_entry_point_twice(desc, sweeps):
    import torch
    d, L, N, W, lo, hi, seed = desc
    V = L ** d
    e_lo, e_hi = -d * N, 0
    nb = e_hi - e_lo + 1
    lnW = workloads.random_log_weights(nb, 21, scale=0.1)
    T = chain.thresholds(d, e_lo, e_hi, lnW)
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    t_bits, t_S, t_E = _to_device(occ, S, E)
    t_thr = torch.from_numpy(T.reshape(-1).view(np.int32).copy()).cuda()
    t_H = torch.zeros(nb, dtype=torch.int64, device="cuda")
    with m.Mucal([desc]) as mc:
        mc.set_weights(0, lnW)
        np.testing.assert_array_equal(mc.thresholds(0), T)
        for it in range(2):
            mc.run_iteration(sweeps, it)
            H_ref = mc.histogram(0)
            _call(desc, sweeps, it, t_bits, t_S, t_E, t_thr, t_H)
            torch.cuda.synchronize()
            hist, _ = chain.run_walkers(d, L, N, seed, it, sweeps * N, e_lo, e_hi, T, S, occ, E)
            H = t_H.cpu().numpy()
            np.testing.assert_array_equal(H, hist.sum(axis=0))
            np.testing.assert_array_equal(H, H_ref)
            assert int(H.sum()) == W * sweeps * N
            bits, S_g, E_g = _from_device(t_bits, t_S, t_E, V)
            np.testing.assert_array_equal(E_g, E)
            np.testing.assert_array_equal(S_g, S)
            np.testing.assert_array_equal(bits, _pack_bits(occ))
            for w in (0, W // 2, W - 1):
                g_occ, g_S, g_E = mc.walker_state(0, w)
                assert g_E == E[w]
                np.testing.assert_array_equal(g_S, S[w])
                np.testing.assert_array_equal(g_occ, occ[w])


def _bad_input_case(corrupt):
    import torch
    desc = (2, 16, 40, 64, 0, 0, 3)
    d, L, N, W, lo, hi, seed = desc
    V = L ** d
    nb = d * N + 1
    T = chain.thresholds(d, -d * N, 0, np.zeros(nb))
    S, occ, E = chain.init_walkers(d, L, N, W, seed)
    corrupt(S, E, V, nb)
    t_bits, t_S, t_E = _to_device(occ, S, E)
    t_thr = torch.from_numpy(T.reshape(-1).view(np.int32).copy()).cuda()
    t_H = torch.zeros(nb, dtype=torch.int64, device="cuda")
    before = _from_device(t_bits, t_S, t_E, V)
    with pytest.raises(m.MucalError) as ei:
        _call(desc, 10, 0, t_bits, t_S, t_E, t_thr, t_H)
    torch.cuda.synchronize()
    after = _from_device(t_bits, t_S, t_E, V)
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x, y)
    assert ei.value.code == m.MUCAL_ERR_INVALID_ARG
    return str(ei.value)


def test_noalloc_rejects_energy_outside_window():
    def corrupt(S, E, V, nb):
        E[5] = 1                      # above e_hi = 0
    assert "outside the window" in _bad_input_case(corrupt)


def test_noalloc_rejects_list_entry_beyond_lattice():
    def corrupt(S, E, V, nb):
        S[7, 3] = V                   # not a site of the 16 x 16 lattice
    assert "not a lattice site" in _bad_input_case(corrupt)


def test_noalloc_runs_after_a_rejected_call():
    """A rejected call leaves the shared scratch usable: the next valid call
    on the same buffers matches the oracle."""
    import torch

    def corrupt(S, E, V, nb):
        E[0] = -10 ** 6
    _bad_input_case(corrupt)
    test_noalloc_matches_oracle_and_regular_entry_point_twice(*CASES[0])
    torch.cuda.synchronize()
