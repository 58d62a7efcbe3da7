"""Host-side checks of the C ABI: the library builds, loads, exports every
function declared in include/mucal.h, and rejects bad arguments before it
touches a device.  No compute call runs here."""
import os
import re

import pytest

from paper_1401_4076_gb300 import mucal as m

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    return m.load_library()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mucal_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "mucal_init_systems" in names and "mucal_run_iteration" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(m.EXPORTED) <= names


def test_version_string(lib):
    assert "sm_103a" in m.mucal_version()


@pytest.mark.parametrize("desc,msg", [
    ((4, 8, 4, 1, 0, 0, 0), "d must be"),
    ((2, 2, 2, 1, 0, 0, 0), "L must be"),
    ((2, 8, 0, 1, 0, 0, 0), "0 < N"),
    ((2, 8, 64, 1, 0, 0, 0), "0 < N"),
    ((2, 8, 4, 0, 0, 0, 0), "n_walkers"),
    ((2, 8, 4, 1, -9, 0, 0), "window"),
    ((2, 8, 4, 1, -4, -5, 0), "window"),
])
def test_invalid_descriptors_rejected_before_device_use(lib, desc, msg):
    with pytest.raises(m.MucalError) as ei:
        m.mucal_init_systems([desc])
    assert ei.value.code == m.MUCAL_ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(m.MucalError) as ei:
        m.mucal_init_systems([(2, 8, 4, 2, 0, 0, 0)])
    assert ei.value.code == m.MUCAL_ERR_NO_DEVICE


def test_calls_on_null_context_fail(lib):
    assert lib.mucal_run_iteration(None, 1, 0) == m.MUCAL_ERR_INVALID_ARG
    assert lib.mucal_set_weights(None, 0, None, 0) == m.MUCAL_ERR_INVALID_ARG


@pytest.mark.parametrize("desc,msg", [
    ((2, 64, 100, (1 << 20) + 1, 0, 0, 0), "n_walkers"),
    # ceil(8000 / 32) * 19201 bins > 2^22 histogram entries of the fixed scratch
    ((3, 40, 6400, 8000, 0, 0, 0), "histogram entries"),
    ((2, 16, 300, 8, 0, 0, 0), "0 < N"),
])
def test_noalloc_limits_rejected_before_device_use(lib, desc, msg):
    """The allocation-free call rejects sizes beyond its fixed scratch on the
    host, before it looks for a device (the pointers are never touched)."""
    with pytest.raises(m.MucalError) as ei:
        m.mucal_run_walkers_noalloc(desc, 1, 0, 16, 16, 16, 16, 16, None)
    assert ei.value.code == m.MUCAL_ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_noalloc_null_buffer_rejected(lib):
    with pytest.raises(m.MucalError) as ei:
        m.mucal_run_walkers_noalloc((2, 8, 4, 2, 0, 0, 0), 1, 0, 16, 0, 16, 16, 16, None)
    assert ei.value.code == m.MUCAL_ERR_INVALID_ARG
