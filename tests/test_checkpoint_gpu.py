"""Checkpoint and resume through the C ABI (GPU), and host-side rejection of
corrupted checkpoints (the fault is injected into the host buffer; nothing
invalid reaches the device)."""
import numpy as np
import pytest

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


DESCS = [(2, 24, 60, 70, 0, 0, 5), (3, 10, 90, 33, 0, 0, 900)]


def test_resume_is_bit_exact():
    with m.Mucal(DESCS) as a:
        for it in range(2):
            a.run_iteration(30, it)
            for s in range(2):
                a.update_weights(s)
        cks = [a.checkpoint(s) for s in range(2)]
        a.run_iteration(30, 2)
        Ha = [a.histogram(s) for s in range(2)]
        Wa = [a.update_weights(s)[0] for s in range(2)]
        Ea = [a.walker_state(s, 3)[2] for s in range(2)]
    with m.Mucal(DESCS) as b:
        for s in range(2):
            b.restore(s, cks[s])
        b.run_iteration(30, 2)
        for s in range(2):
            np.testing.assert_array_equal(b.histogram(s), Ha[s])
            np.testing.assert_array_equal(b.update_weights(s)[0], Wa[s])
            assert b.walker_state(s, 3)[2] == Ea[s]


def test_corrupted_checkpoints_are_rejected():
    with m.Mucal(DESCS[:1]) as a:
        a.run_iteration(10, 0)
        ck = a.checkpoint(0)
        H_before = a.histogram(0)
        info = a.info[0]
        W, V, words = info["n_walkers"], info["V"], (info["V"] + 31) // 32
        hdr = len(ck) - (W * words * 4 + W * V * 2 + W * 4 + info["n_bins"] * 17)
        bad = ck.copy()                     # a list entry off the lattice
        bad[hdr + W * words * 4: hdr + W * words * 4 + 2] = np.frombuffer(
            np.uint16(V + 5).tobytes(), np.uint8)
        with pytest.raises(m.MucalError) as ei:
            a.restore(0, bad)
        assert ei.value.code == m.MUCAL_ERR_INVALID_ARG
        bad = ck.copy()                     # an energy outside the window
        off = hdr + W * words * 4 + W * V * 2
        bad[off: off + 4] = np.frombuffer(np.int32(5).tobytes(), np.uint8)
        with pytest.raises(m.MucalError):
            a.restore(0, bad)
        bad = ck.copy()                     # wrong magic
        bad[0] ^= 0xFF
        with pytest.raises(m.MucalError):
            a.restore(0, bad)
        with pytest.raises(m.MucalError):   # wrong size
            a.restore(0, ck[:-1])
        # nothing was changed: the state still continues as before
        a.restore(0, ck)
        a.run_iteration(10, 0)
        assert a.histogram(0).sum() == H_before.sum()


def test_allocation_failure_is_reported_cleanly():
    """A system far larger than the device: the allocation fails inside the
    library, which returns MUCAL_ERR_OOM and frees what it had taken."""
    huge = (2, 1024, 100, 1 << 22, 0, 0, 0)      # bitsets alone would need 512 GiB
    with pytest.raises(m.MucalError) as ei:
        m.Mucal([huge])
    assert ei.value.code == m.MUCAL_ERR_OOM
    with m.Mucal([(2, 8, 10, 4, 0, 0, 1)]) as ok:    # the device is still usable
        ok.run_iteration(5, 0)
        assert ok.histogram(0).sum() == 4 * 5 * 10
