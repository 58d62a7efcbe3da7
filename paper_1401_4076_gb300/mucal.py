"""Python binding of libmucal (ctypes, argument marshalling only).

The functions carry the names of the C ABI in ``include/mucal.h``; every step
of the simulation runs inside the library (CUDA kernels and its host-side
double-precision weight update).  There is no CPU fallback: loading fails
loudly if the compiled library is missing, and ``mucal_init_systems`` raises
if no CUDA device is usable.

``Mucal`` is a small convenience wrapper holding one context.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmucal.so")

MUCAL_OK = 0
MUCAL_ERR_INVALID_ARG = -1
MUCAL_ERR_CUDA = -2
MUCAL_ERR_OOM = -3
MUCAL_ERR_NO_DEVICE = -4
MUCAL_ERR_NOT_READY = -5
MUCAL_ERR_STATE = -6
MUCAL_FLAG_PER_WALKER_HIST = 0x1
MUCAL_SCHEME_SIMPLE = 0
MUCAL_SCHEME_RECURSIVE = 1
MUCAL_SCHEME_EXTRAPOLATE = 0x10
MUCAL_KERNEL_THREAD = 0
MUCAL_KERNEL_GROUP = 1
MUCAL_KERNEL_FIELD = 2

EXPORTED = [
    "mucal_init_systems", "mucal_destroy", "mucal_last_error", "mucal_set_weights",
    "mucal_get_weights", "mucal_get_thresholds", "mucal_set_launch_config",
    "mucal_get_launch_config", "mucal_run_iteration", "mucal_get_histogram",
    "mucal_update_weights", "mucal_set_target_window", "mucal_get_walker_state",
    "mucal_get_system_info", "mucal_get_stats", "mucal_histogram_device_ptr", "mucal_version",
    "mucal_mlp_param_count", "mucal_mlp_create", "mucal_mlp_destroy", "mucal_mlp_last_error",
    "mucal_mlp_get_params", "mucal_mlp_forward", "mucal_mlp_gradients", "mucal_mlp_train",
    "mucal_run_walkers_noalloc", "mucal_run_walkers_noalloc_error",
    "mucal_checkpoint_size", "mucal_checkpoint_save", "mucal_checkpoint_load",
    "mucal_reweight", "mucal_reweight_system", "mucal_measure_droplets", "mucal_get_droplet_stats",
    "mucal_get_largest_droplets", "mucal_reset_droplet_stats", "mucal_droplet_delta",
    "mucal_droplet_lambda", "mucal_replica_exchange", "mucal_set_tunnel_window",
    "mucal_get_tunnel_counts", "mucal_reset_tunnel_counts", "mucal_set_graph_mode",
    "mucal_mlp_forward_tcgen05", "mucal_mlp_use_tcgen05", "mucal_multi_histogram",
    "mucal_ising_constant", "mucal_set_histogram", "mucal_get_launch_occupancy",
    "mucal_weight_update", "mucal_ln_omega", "mucal_ln_omega_normalise",
]


class mucal_system_desc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32), ("N", ctypes.c_int32),
                ("n_walkers", ctypes.c_int32), ("e_lo", ctypes.c_int32), ("e_hi", ctypes.c_int32),
                ("seed_base", ctypes.c_uint64)]


class mucal_launch_config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("lanes_per_walker", ctypes.c_int32),
                ("walkers_per_block", ctypes.c_int32), ("bits_in_smem", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("thr_window", ctypes.c_int32),
                ("multi_commit", ctypes.c_int32)]


class mucal_system_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32), ("N", ctypes.c_int32),
                ("n_walkers", ctypes.c_int32), ("e_lo", ctypes.c_int32), ("e_hi", ctypes.c_int32),
                ("V", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("width", ctypes.c_int32),
                ("index_bytes", ctypes.c_int32), ("seed_base", ctypes.c_uint64)]


class mucal_stats(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_uint64), ("accepts", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_double), ("iteration_ms", ctypes.c_double),
                ("walker_launches", ctypes.c_uint64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmucal.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmucal.so not found at {path}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "mucal_init_systems": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(mucal_system_desc),
                                              I32, P, U32]),
        "mucal_destroy": (None, [P]),
        "mucal_last_error": (ctypes.c_char_p, [P]),
        "mucal_set_weights": (ctypes.c_int, [P, I32, P, I32]),
        "mucal_get_weights": (ctypes.c_int, [P, I32, P, I32]),
        "mucal_get_thresholds": (ctypes.c_int, [P, I32, P, I64]),
        "mucal_set_launch_config": (ctypes.c_int, [P, ctypes.POINTER(mucal_launch_config)]),
        "mucal_get_launch_config": (ctypes.c_int, [P, ctypes.POINTER(mucal_launch_config)]),
        "mucal_run_iteration": (ctypes.c_int, [P, I64, U32]),
        "mucal_get_histogram": (ctypes.c_int, [P, I32, P, I32, P]),
        "mucal_update_weights": (ctypes.c_int, [P, I32, I32, P, P]),
        "mucal_set_target_window": (ctypes.c_int, [P, I32, I32, I32]),
        "mucal_get_walker_state": (ctypes.c_int, [P, I32, I32, P, P, P]),
        "mucal_get_system_info": (ctypes.c_int, [P, I32, ctypes.POINTER(mucal_system_info)]),
        "mucal_get_stats": (ctypes.c_int, [P, I32, ctypes.POINTER(mucal_stats)]),
        "mucal_histogram_device_ptr": (ctypes.c_int, [P, I32, ctypes.POINTER(P)]),
        "mucal_version": (ctypes.c_char_p, []),
        "mucal_mlp_param_count": (ctypes.c_int, []),
        "mucal_mlp_create": (ctypes.c_int, [ctypes.POINTER(P), P, I64, P]),
        "mucal_mlp_destroy": (None, [P]),
        "mucal_mlp_last_error": (ctypes.c_char_p, [P]),
        "mucal_mlp_get_params": (ctypes.c_int, [P, P, I64, I32]),
        "mucal_mlp_forward": (ctypes.c_int, [P, P, I64, P]),
        "mucal_mlp_gradients": (ctypes.c_int, [P, P, P, I64, P, P]),
        "mucal_mlp_train": (ctypes.c_int, [P, P, P, I64, I32, ctypes.c_float, P]),
        "mucal_run_walkers_noalloc": (ctypes.c_int, [ctypes.POINTER(mucal_system_desc), I64, U32,
                                                     P, P, P, P, P, P]),
        "mucal_run_walkers_noalloc_error": (ctypes.c_char_p, []),
        "mucal_checkpoint_size": (ctypes.c_int, [P, I32, ctypes.POINTER(I64)]),
        "mucal_checkpoint_save": (ctypes.c_int, [P, I32, P, I64]),
        "mucal_checkpoint_load": (ctypes.c_int, [P, I32, P, I64]),
        "mucal_reweight": (ctypes.c_int, [P, P, I32, I32, P, I32, P, I32, P, P, P]),
        "mucal_reweight_system": (ctypes.c_int, [P, I32, P, I32, P, I32, P, P, P]),
        "mucal_measure_droplets": (ctypes.c_int, [P]),
        "mucal_get_droplet_stats": (ctypes.c_int, [P, I32, P, P, P, I32]),
        "mucal_get_largest_droplets": (ctypes.c_int, [P, I32, P, I32]),
        "mucal_reset_droplet_stats": (ctypes.c_int, [P]),
        "mucal_droplet_delta": (ctypes.c_int, [I32, I64, I64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, P, P]),
        "mucal_droplet_lambda": (ctypes.c_int, [I32, ctypes.c_double, P]),
        "mucal_replica_exchange": (ctypes.c_int, [P, P, I32, U32, I32, P]),
        "mucal_set_tunnel_window": (ctypes.c_int, [P, I32, I32, I32]),
        "mucal_get_tunnel_counts": (ctypes.c_int, [P, I32, P, P, P]),
        "mucal_reset_tunnel_counts": (ctypes.c_int, [P]),
        "mucal_set_graph_mode": (ctypes.c_int, [P, I32]),
        "mucal_mlp_forward_tcgen05": (ctypes.c_int, [P, P, I64, P]),
        "mucal_mlp_use_tcgen05": (ctypes.c_int, [P, I32]),
        "mucal_multi_histogram": (ctypes.c_int, [P, P, I32, I32, I32, ctypes.c_double, P, P]),
        "mucal_ising_constant": (ctypes.c_int, [I32, I64, I64, ctypes.c_double, P]),
        "mucal_set_histogram": (ctypes.c_int, [P, I32, P, I32]),
        "mucal_get_launch_occupancy": (ctypes.c_int, [P, P, P]),
        "mucal_weight_update": (ctypes.c_int, [I32, I32, P, P, P, P, I32, I32, P]),
        "mucal_ln_omega": (ctypes.c_int, [P, P, I32, I64, I64, P]),
        "mucal_ln_omega_normalise": (ctypes.c_int, [P, I32, I64, I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MucalError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mucal error {code}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != MUCAL_OK:
        msg = load_library().mucal_last_error(ctx)
        raise MucalError(rc, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data


# --------------------------------------------------------------------------
# C ABI, one function per export (same names, numpy arrays for buffers).
# --------------------------------------------------------------------------

def mucal_init_systems(systems, cuda_stream=None, flags=0):
    """systems: list of dicts/tuples (d, L, N, n_walkers, e_lo, e_hi, seed_base)."""
    lib = load_library()
    arr = (mucal_system_desc * len(systems))()
    for i, s in enumerate(systems):
        if isinstance(s, dict):
            s = (s["d"], s["L"], s["N"], s["n_walkers"], s.get("e_lo", 0), s.get("e_hi", 0),
                 s.get("seed_base", 0))
        arr[i] = mucal_system_desc(*s)
    ctx = ctypes.c_void_p()
    rc = lib.mucal_init_systems(ctypes.byref(ctx), arr, len(systems), cuda_stream, flags)
    _check(rc, None)
    return ctx


def mucal_destroy(ctx):
    load_library().mucal_destroy(ctx)


def mucal_last_error(ctx):
    m = load_library().mucal_last_error(ctx)
    return m.decode() if m else ""


def mucal_set_weights(ctx, sys, lnW):
    w = np.ascontiguousarray(lnW, dtype=np.float64)
    _check(load_library().mucal_set_weights(ctx, sys, _ptr(w), w.size), ctx)


def mucal_get_weights(ctx, sys, n_bins):
    out = np.zeros(n_bins, dtype=np.float64)
    _check(load_library().mucal_get_weights(ctx, sys, _ptr(out), n_bins), ctx)
    return out


def mucal_get_thresholds(ctx, sys, n_bins, width):
    T = np.zeros((n_bins, width), dtype=np.uint32)
    _check(load_library().mucal_get_thresholds(ctx, sys, _ptr(T), T.size), ctx)
    return T


def mucal_set_launch_config(ctx, kernel=MUCAL_KERNEL_THREAD, lanes_per_walker=1,
                            walkers_per_block=32, bits_in_smem=1, persistent=0, thr_window=1,
                            multi_commit=0):
    cfg = mucal_launch_config(kernel, lanes_per_walker, walkers_per_block, bits_in_smem,
                              int(persistent), int(thr_window), int(multi_commit))
    _check(load_library().mucal_set_launch_config(ctx, ctypes.byref(cfg)), ctx)


def mucal_get_launch_config(ctx):
    cfg = mucal_launch_config()
    _check(load_library().mucal_get_launch_config(ctx, ctypes.byref(cfg)), ctx)
    return {"kernel": cfg.kernel, "lanes_per_walker": cfg.lanes_per_walker,
            "walkers_per_block": cfg.walkers_per_block, "bits_in_smem": cfg.bits_in_smem,
            "persistent": cfg.persistent, "thr_window": cfg.thr_window,
            "multi_commit": cfg.multi_commit}


def mucal_set_graph_mode(ctx, enable):
    _check(load_library().mucal_set_graph_mode(ctx, 1 if enable else 0), ctx)


def mucal_run_iteration(ctx, sweeps, iteration):
    _check(load_library().mucal_run_iteration(ctx, int(sweeps), int(iteration) & 0xFFFFFFFF), ctx)


def mucal_get_histogram(ctx, sys, n_bins, per_walker_shape=None):
    H = np.zeros(n_bins, dtype=np.int64)
    pw = None if per_walker_shape is None else np.zeros(per_walker_shape, dtype=np.int64)
    _check(load_library().mucal_get_histogram(ctx, sys, _ptr(H), n_bins, _ptr(pw)), ctx)
    return H if pw is None else (H, pw)


def mucal_update_weights(ctx, sys, scheme, n_bins):
    lnW = np.zeros(n_bins, dtype=np.float64)
    f = ctypes.c_double()
    _check(load_library().mucal_update_weights(ctx, sys, scheme, _ptr(lnW), ctypes.addressof(f)),
           ctx)
    return lnW, f.value


def mucal_set_target_window(ctx, sys, t_lo, t_hi):
    _check(load_library().mucal_set_target_window(ctx, sys, t_lo, t_hi), ctx)


def mucal_get_walker_state(ctx, sys, walker, V):
    occ = np.zeros(V, dtype=np.uint8)
    S = np.zeros(V, dtype=np.int32)
    E = ctypes.c_int32()
    _check(load_library().mucal_get_walker_state(ctx, sys, walker, _ptr(occ), _ptr(S),
                                                  ctypes.addressof(E)), ctx)
    return occ, S, E.value


def mucal_get_system_info(ctx, sys):
    info = mucal_system_info()
    _check(load_library().mucal_get_system_info(ctx, sys, ctypes.byref(info)), ctx)
    return {f: getattr(info, f) for f, _ in mucal_system_info._fields_}


def mucal_get_stats(ctx, sys):
    st = mucal_stats()
    _check(load_library().mucal_get_stats(ctx, sys, ctypes.byref(st)), ctx)
    return {f: getattr(st, f) for f, _ in mucal_stats._fields_}


def mucal_histogram_device_ptr(ctx, sys):
    p = ctypes.c_void_p()
    _check(load_library().mucal_histogram_device_ptr(ctx, sys, ctypes.byref(p)), ctx)
    return p.value


def mucal_version():
    return load_library().mucal_version().decode()


def mucal_checkpoint_save(ctx, sys):
    """Checkpoint of system sys as a bytes-like numpy uint8 array."""
    lib = load_library()
    n = ctypes.c_int64()
    _check(lib.mucal_checkpoint_size(ctx, sys, ctypes.byref(n)), ctx)
    buf = np.zeros(n.value, dtype=np.uint8)
    _check(lib.mucal_checkpoint_save(ctx, sys, _ptr(buf), buf.size), ctx)
    return buf


def mucal_checkpoint_load(ctx, sys, buf):
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().mucal_checkpoint_load(ctx, sys, _ptr(b), b.size), ctx)


def mucal_run_walkers_noalloc(desc, sweeps, iteration, bits_ptr, S_ptr, E_ptr, thr_ptr, H_ptr,
                              cuda_stream=None):
    """Allocation-free walker update on caller-owned device buffers (raw
    device pointers as ints); see include/mucal.h for layouts and limits."""
    lib = load_library()
    d = mucal_system_desc(*desc)
    rc = lib.mucal_run_walkers_noalloc(ctypes.byref(d), int(sweeps), int(iteration) & 0xFFFFFFFF,
                                       bits_ptr, S_ptr, E_ptr, thr_ptr, H_ptr, cuda_stream)
    if rc != MUCAL_OK:
        raise MucalError(rc, lib.mucal_run_walkers_noalloc_error().decode())


def _f64(a):
    return np.ascontiguousarray(np.atleast_1d(np.asarray(a, dtype=np.float64)))


def _reweight_args(beta, obs, n_bins):
    b = _f64(beta)
    if obs is None:
        o = None
        n_obs = 0
    else:
        o = np.ascontiguousarray(np.atleast_2d(np.asarray(obs, dtype=np.float64)))
        if o.shape[1] != n_bins:
            raise ValueError(f"obs rows must hold n_bins = {n_bins} values")
        n_obs = o.shape[0]
    mE = np.zeros(b.size)
    mE2 = np.zeros(b.size)
    out = np.zeros((b.size, n_obs)) if n_obs else None
    return b, o, n_obs, mE, mE2, out


def mucal_reweight(H, lnW, e_lo, beta, obs=None):
    """(<E>, <E^2>[, obs means]) at each beta from a histogram H sampled with
    lnW (Sec. 3 reweighting); obs: (n_obs, n_bins) microcanonical means, NaN
    where unmeasured."""
    h = np.ascontiguousarray(H, dtype=np.int64)
    w = np.ascontiguousarray(lnW, dtype=np.float64)
    if w.size != h.size:
        raise ValueError("H and lnW differ in length")
    b, o, n_obs, mE, mE2, out = _reweight_args(beta, obs, h.size)
    _check(load_library().mucal_reweight(_ptr(h), _ptr(w), h.size, int(e_lo), _ptr(b), b.size,
                                         _ptr(o), n_obs, _ptr(mE), _ptr(mE2), _ptr(out)), None)
    return (mE, mE2) if out is None else (mE, mE2, out)


def mucal_multi_histogram(H, lnW, max_iter=10000, tol=1e-12):
    """ln Omega (max 0, NaN where unvisited) from histograms H[K][n_bins]
    sampled with lnW[K][n_bins]; returns (ln_omega, passes)."""
    h = np.ascontiguousarray(np.atleast_2d(H), dtype=np.int64)
    w = np.ascontiguousarray(np.atleast_2d(lnW), dtype=np.float64)
    if h.shape != w.shape:
        raise ValueError("H and lnW differ in shape")
    out = np.zeros(h.shape[1])
    it = ctypes.c_int32()
    _check(load_library().mucal_multi_histogram(_ptr(h), _ptr(w), h.shape[0], h.shape[1],
                                                int(max_iter), float(tol), _ptr(out),
                                                ctypes.addressof(it)), None)
    return out, it.value


def mucal_ising_constant(d, V, N, J=1.0):
    c = ctypes.c_double()
    _check(load_library().mucal_ising_constant(int(d), int(V), int(N), float(J),
                                               ctypes.addressof(c)), None)
    return c.value


def mucal_set_histogram(ctx, sys, H):
    """Hand system sys a summed histogram (e.g. the sum over processes) for
    its next weight update."""
    h = np.ascontiguousarray(H, dtype=np.int64)
    _check(load_library().mucal_set_histogram(ctx, sys, _ptr(h), h.size), ctx)


def mucal_get_launch_occupancy(ctx):
    """(resident blocks per SM of the current launch shape, SM count)."""
    b = ctypes.c_int32()
    n = ctypes.c_int32()
    _check(load_library().mucal_get_launch_occupancy(ctx, ctypes.addressof(b),
                                                     ctypes.addressof(n)), ctx)
    return b.value, n.value


class WeightState:
    """Host arrays of one weight iteration (lnW, cumulative visited set,
    accumulated pair weights) for ``mucal_weight_update``."""

    def __init__(self, n_bins, lnW=None):
        self.lnW = np.zeros(n_bins) if lnW is None else np.array(lnW, dtype=np.float64)
        self.visited = np.zeros(n_bins, dtype=np.uint8)
        self.pacc = np.zeros(n_bins)


def mucal_weight_update(state, H, scheme=MUCAL_SCHEME_RECURSIVE, target=None):
    """One weight update of Sec. 2 on a WeightState, in place; returns the
    flatness.  target: (t_lo, t_hi) in bins, or None for the visited range."""
    h = np.ascontiguousarray(H, dtype=np.int64)
    n = h.size
    if state.lnW.size != n:
        raise ValueError("H and the weight state differ in length")
    t_lo, t_hi = (-1, -1) if target is None else (int(target[0]), int(target[1]))
    f = ctypes.c_double()
    _check(load_library().mucal_weight_update(int(scheme), n, _ptr(h), _ptr(state.lnW),
                                              _ptr(state.visited), _ptr(state.pacc), t_lo, t_hi,
                                              ctypes.addressof(f)), None)
    return f.value


def mucal_ln_omega(H, lnW, V, N):
    """ln Omega(E) = ln H - lnW on visited bins, normalised to C(V, N) states."""
    h = np.ascontiguousarray(H, dtype=np.int64)
    w = np.ascontiguousarray(lnW, dtype=np.float64)
    if h.size != w.size:
        raise ValueError("H and lnW differ in length")
    out = np.zeros(h.size)
    _check(load_library().mucal_ln_omega(_ptr(h), _ptr(w), h.size, int(V), int(N), _ptr(out)),
           None)
    return out


def mucal_ln_omega_normalise(ln_omega, V, N):
    """Shift finite entries so that their exponentials sum to C(V, N)."""
    out = np.array(ln_omega, dtype=np.float64)
    _check(load_library().mucal_ln_omega_normalise(_ptr(out), out.size, int(V), int(N)), None)
    return out


def mucal_reweight_system(ctx, sys, n_bins, beta, obs=None):
    b, o, n_obs, mE, mE2, out = _reweight_args(beta, obs, n_bins)
    _check(load_library().mucal_reweight_system(ctx, sys, _ptr(b), b.size, _ptr(o), n_obs,
                                                _ptr(mE), _ptr(mE2), _ptr(out)), ctx)
    return (mE, mE2) if out is None else (mE, mE2, out)


def mucal_set_tunnel_window(ctx, sys, e_min, e_max):
    _check(load_library().mucal_set_tunnel_window(ctx, sys, int(e_min), int(e_max)), ctx)


def mucal_get_tunnel_counts(ctx, sys, n_walkers):
    """(total, per-walker uint32 counts, per-walker uint8 states)."""
    tot = ctypes.c_int64()
    cnt = np.zeros(n_walkers, dtype=np.uint32)
    st = np.zeros(n_walkers, dtype=np.uint8)
    _check(load_library().mucal_get_tunnel_counts(ctx, sys, ctypes.addressof(tot), _ptr(cnt),
                                                  _ptr(st)), ctx)
    return tot.value, cnt, st


def mucal_reset_tunnel_counts(ctx):
    _check(load_library().mucal_reset_tunnel_counts(ctx), ctx)


def mucal_replica_exchange(ctx, beta, round_, parity):
    """Exchange configurations between neighbouring systems of a tempering
    ladder; returns the accepted exchanges per pair (int64[n_sys - 1])."""
    b = _f64(beta)
    acc = np.zeros(max(b.size - 1, 1), dtype=np.int64)
    _check(load_library().mucal_replica_exchange(ctx, _ptr(b), b.size, int(round_) & 0xFFFFFFFF,
                                                 int(parity), _ptr(acc)), ctx)
    return acc[: b.size - 1]


def mucal_measure_droplets(ctx):
    _check(load_library().mucal_measure_droplets(ctx), ctx)


def mucal_get_droplet_stats(ctx, sys, n_bins):
    """(count, sum V_D, sum V_D^2) per energy bin, int64 arrays."""
    out = [np.zeros(n_bins, dtype=np.int64) for _ in range(3)]
    _check(load_library().mucal_get_droplet_stats(ctx, sys, *[_ptr(a) for a in out], n_bins), ctx)
    return tuple(out)


def mucal_get_largest_droplets(ctx, sys, n_walkers):
    out = np.zeros(n_walkers, dtype=np.int32)
    _check(load_library().mucal_get_largest_droplets(ctx, sys, _ptr(out), n_walkers), ctx)
    return out


def mucal_reset_droplet_stats(ctx):
    _check(load_library().mucal_reset_droplet_stats(ctx), ctx)


def mucal_droplet_delta(d, V, N, rho0, kappa_hat, tau_W):
    """(Delta, V_L) of Eqs. 8 and 10."""
    delta = ctypes.c_double()
    vl = ctypes.c_double()
    _check(load_library().mucal_droplet_delta(int(d), int(V), int(N), float(rho0), float(kappa_hat),
                                              float(tau_W), ctypes.addressof(delta),
                                              ctypes.addressof(vl)), None)
    return delta.value, vl.value


def mucal_droplet_lambda(d, Delta):
    lam = ctypes.c_double()
    _check(load_library().mucal_droplet_lambda(int(d), float(Delta), ctypes.addressof(lam)), None)
    return lam.value


# --------------------------------------------------------------------------
# Convenience wrapper.
# --------------------------------------------------------------------------

@dataclass
class SystemDesc:
    d: int
    L: int
    N: int
    n_walkers: int
    e_lo: int = 0
    e_hi: int = 0
    seed_base: int = 0

    def as_tuple(self):
        return (self.d, self.L, self.N, self.n_walkers, self.e_lo, self.e_hi, self.seed_base)


class Mucal:
    """One library context over several systems, with numpy-returning helpers."""

    def __init__(self, systems, cuda_stream=None, per_walker_hist=False):
        descs = [s.as_tuple() if isinstance(s, SystemDesc) else s for s in systems]
        flags = MUCAL_FLAG_PER_WALKER_HIST if per_walker_hist else 0
        self.ctx = mucal_init_systems(descs, cuda_stream, flags)
        self.info = [mucal_get_system_info(self.ctx, i) for i in range(len(descs))]

    def close(self):
        if self.ctx is not None:
            mucal_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_weights(self, sys, lnW):
        mucal_set_weights(self.ctx, sys, lnW)

    def weights(self, sys):
        return mucal_get_weights(self.ctx, sys, self.info[sys]["n_bins"])

    def thresholds(self, sys):
        i = self.info[sys]
        return mucal_get_thresholds(self.ctx, sys, i["n_bins"], i["width"])

    def set_launch(self, **kw):
        mucal_set_launch_config(self.ctx, **kw)

    def launch(self):
        return mucal_get_launch_config(self.ctx)

    def run_iteration(self, sweeps, iteration):
        mucal_run_iteration(self.ctx, sweeps, iteration)

    def histogram(self, sys, per_walker=False):
        i = self.info[sys]
        shape = (i["n_walkers"], i["n_bins"]) if per_walker else None
        return mucal_get_histogram(self.ctx, sys, i["n_bins"], shape)

    def update_weights(self, sys, scheme=MUCAL_SCHEME_RECURSIVE):
        return mucal_update_weights(self.ctx, sys, scheme, self.info[sys]["n_bins"])

    def set_target_window(self, sys, t_lo, t_hi):
        mucal_set_target_window(self.ctx, sys, t_lo, t_hi)

    def set_histogram(self, sys, H):
        mucal_set_histogram(self.ctx, sys, H)

    def occupancy(self):
        return mucal_get_launch_occupancy(self.ctx)

    def walker_state(self, sys, walker):
        return mucal_get_walker_state(self.ctx, sys, walker, self.info[sys]["V"])

    def stats(self, sys=0):
        return mucal_get_stats(self.ctx, sys)

    def checkpoint(self, sys=0):
        return mucal_checkpoint_save(self.ctx, sys)

    def restore(self, sys, buf):
        mucal_checkpoint_load(self.ctx, sys, buf)

    def reweight(self, sys, beta, obs=None):
        return mucal_reweight_system(self.ctx, sys, self.info[sys]["n_bins"], beta, obs)

    def set_graph_mode(self, enable=True):
        mucal_set_graph_mode(self.ctx, enable)

    def set_tunnel_window(self, sys, e_min, e_max):
        mucal_set_tunnel_window(self.ctx, sys, e_min, e_max)

    def tunnel_counts(self, sys):
        return mucal_get_tunnel_counts(self.ctx, sys, self.info[sys]["n_walkers"])

    def reset_tunnel_counts(self):
        mucal_reset_tunnel_counts(self.ctx)

    def replica_exchange(self, beta, round_, parity):
        return mucal_replica_exchange(self.ctx, beta, round_, parity)

    def measure_droplets(self):
        mucal_measure_droplets(self.ctx)

    def droplet_stats(self, sys):
        return mucal_get_droplet_stats(self.ctx, sys, self.info[sys]["n_bins"])

    def largest_droplets(self, sys):
        return mucal_get_largest_droplets(self.ctx, sys, self.info[sys]["n_walkers"])

    def reset_droplet_stats(self):
        mucal_reset_droplet_stats(self.ctx)


# --------------------------------------------------------------------------
# Weight-seeding network.
# --------------------------------------------------------------------------

def _mlp_check(rc, mlp=None):
    if rc != MUCAL_OK:
        msg = load_library().mucal_mlp_last_error(mlp)
        raise MucalError(rc, msg.decode() if msg else "")


def mucal_mlp_param_count():
    return int(load_library().mucal_mlp_param_count())


def mucal_mlp_create(params, cuda_stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = ctypes.c_void_p()
    _mlp_check(load_library().mucal_mlp_create(ctypes.byref(h), _ptr(p), p.size, cuda_stream))
    return h


def mucal_mlp_destroy(mlp):
    load_library().mucal_mlp_destroy(mlp)


def mucal_mlp_get_params(mlp, rounded=False):
    out = np.zeros(mucal_mlp_param_count(), dtype=np.float32)
    _mlp_check(load_library().mucal_mlp_get_params(mlp, _ptr(out), out.size, int(bool(rounded))), mlp)
    return out


def mucal_mlp_forward(mlp, X):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 4)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _mlp_check(load_library().mucal_mlp_forward(mlp, _ptr(X), X.shape[0], _ptr(y)), mlp)
    return y


def mucal_mlp_forward_tcgen05(mlp, X):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 4)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _mlp_check(load_library().mucal_mlp_forward_tcgen05(mlp, _ptr(X), X.shape[0], _ptr(y)), mlp)
    return y


def mucal_mlp_gradients(mlp, X, t):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 4)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(mucal_mlp_param_count(), dtype=np.float32)
    loss = ctypes.c_float()
    _mlp_check(load_library().mucal_mlp_gradients(mlp, _ptr(X), _ptr(t), X.shape[0],
                                                   ctypes.addressof(loss), _ptr(g)), mlp)
    return loss.value, g


def mucal_mlp_train(mlp, X, t, steps, lr):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, 4)
    t = np.ascontiguousarray(t, dtype=np.float32)
    loss = ctypes.c_float()
    _mlp_check(load_library().mucal_mlp_train(mlp, _ptr(X), _ptr(t), X.shape[0], int(steps),
                                               float(lr), ctypes.addressof(loss)), mlp)
    return loss.value


MLP_LAYOUT = (("W1", (128, 4)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
              ("W3", (1, 128)), ("b3", (1,)))


def mlp_unflatten(vec):
    """Split the flat parameter vector into named arrays (views)."""
    out, off = {}, 0
    for name, shape in MLP_LAYOUT:
        n = int(np.prod(shape))
        out[name] = np.asarray(vec[off: off + n]).reshape(shape)
        off += n
    return out


def mlp_flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float32).reshape(-1)
                           for name, _ in MLP_LAYOUT])


class Mlp:
    """The seeding network on the GPU (one handle)."""

    def __init__(self, params, cuda_stream=None):
        self.h = mucal_mlp_create(params, cuda_stream)

    def close(self):
        if self.h is not None:
            mucal_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def params(self, rounded=False):
        return mucal_mlp_get_params(self.h, rounded)

    def forward(self, X):
        return mucal_mlp_forward(self.h, X)

    def forward_tcgen05(self, X):
        return mucal_mlp_forward_tcgen05(self.h, X)

    def use_tcgen05(self, enable=True):
        _mlp_check(load_library().mucal_mlp_use_tcgen05(self.h, 1 if enable else 0), self.h)

    def gradients(self, X, t):
        return mucal_mlp_gradients(self.h, X, t)

    def train(self, X, t, steps, lr):
        return mucal_mlp_train(self.h, X, t, steps, lr)
