"""Compile and load the C part of the oracle (test infrastructure only).

The shared object is built with gcc into ``oracle/_build/`` next to this file;
nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mucal_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libmucal_oracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ``mucal_oracle.c`` with gcc (OpenMP over walkers) if stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(lib):
    c = ctypes
    i32, i64, u32, u64, dbl = c.c_int32, c.c_int64, c.c_uint32, c.c_uint64, c.c_double
    P = c.c_void_p
    sig = {
        "orc_philox4x32_10": (None, [P, P, P]),
        "orc_philox_batch": (None, [i64, P, P, P]),
        "orc_volume": (i64, [c.c_int, c.c_int]),
        "orc_neighbours": (None, [c.c_int, c.c_int, i64, P]),
        "orc_energy": (i64, [c.c_int, c.c_int, P]),
        "orc_delta_e": (c.c_int, [c.c_int, c.c_int, P, i64, i64]),
        "orc_init_walker": (None, [c.c_int, c.c_int, c.c_int, u64, P, P, P]),
        "orc_init_walkers": (None, [c.c_int, c.c_int, c.c_int, i64, u64, P, P, P]),
        "orc_thresholds": (None, [c.c_int, c.c_int, c.c_int, P, P]),
        "orc_run_walker": (c.c_int, [c.c_int, c.c_int, c.c_int, u64, u32, i64, c.c_int,
                                     c.c_int, P, P, P, P, P, P]),
        "orc_run_walkers": (i64, [c.c_int, c.c_int, c.c_int, i64, u64, u32, i64, c.c_int,
                                  c.c_int, P, P, P, P, P, P]),
        "orc_num_threads": (c.c_int, []),
        "orc_enumerate": (i64, [c.c_int, c.c_int, c.c_int, P]),
        "orc_energy_mask": (i64, [c.c_int, c.c_int, u64]),
        "orc_delta_e_mask": (c.c_int, [c.c_int, c.c_int, u64, i64, i64]),
        "orc_ising_fixed_m": (c.c_int, [c.c_int, c.c_int, c.c_int, u64, dbl, i64, i64, P, P]),
        "orc_largest_cluster": (i64, [c.c_int, c.c_int, P]),
        "orc_replica_exchange": (None, [c.c_int, i64, i64, P, P, u32, c.c_int, P, P, P, P]),
        "orc_run_walkers_tunnel": (i64, [c.c_int, c.c_int, c.c_int, i64, u64, u32, i64, c.c_int,
                                         c.c_int, P, P, P, P, P, c.c_int, c.c_int, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _ = (i32,)
    return lib


def load_oracle():
    """Return the ctypes handle of the compiled oracle, building it first."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build_oracle()))
    return _lib
