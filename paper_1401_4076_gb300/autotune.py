"""Launch-shape autotuner for the walker update.

For a set of systems it times every candidate launch shape: kernel (one
thread per walker, G lanes per walker on the occupation bits, or G lanes per
walker on a field of neighbour counts), walkers per block, whether the
occupation bitsets are staged in shared memory, and (for the finalists)
whether the launch is persistent.  All candidates compute the
identical chain (the group kernel commits attempts in order), so only speed
differs.  Timing runs on a scratch context whose walkers use other seeds, so
the caller's chains are not advanced.  The acceptance rate changes which
shape wins, so the caller passes the weights it will run with.
"""
from __future__ import annotations

import json
import statistics

from . import mucal as m


def candidates(max_threads: int = 1024):
    """Launch shapes to try.  Block sizes include odd multiples of a warp so
    that a one-wave launch can match walkers to SMs when shared memory limits
    the blocks per SM."""
    out = []
    for wpb in (2, 4, 6, 8, 12, 16, 27, 32, 64):
        for smem in (1, 0):
            out.append(dict(kernel=m.MUCAL_KERNEL_THREAD, lanes_per_walker=1,
                            walkers_per_block=wpb, bits_in_smem=smem))
    for g in (4, 8, 16, 32):
        for threads in (64, 96, 128, 160, 192, 224, 256, 384, 512):
            wpb = threads // g
            if wpb < 1 or threads > max_threads:
                continue
            for smem in (1, 0):
                out.append(dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=g,
                                walkers_per_block=wpb, bits_in_smem=smem))
            # the field lives in shared memory; shapes it does not fit are
            # rejected by the library and skipped
            out.append(dict(kernel=m.MUCAL_KERNEL_FIELD, lanes_per_walker=g,
                            walkers_per_block=wpb, bits_in_smem=1))
    return out


def _time(mc, cfg, sweeps, repeats, it):
    mc.set_launch(**cfg)
    mc.run_iteration(sweeps, it)      # warm-up of this shape
    it += 1
    times = []
    for _ in range(repeats):
        mc.run_iteration(sweeps, it)
        it += 1
        times.append(mc.stats(0)["kernel_ms"])
    return statistics.median(times), it


def autotune(systems, lnW=None, sweeps: int = 20, repeats: int = 3, cuda_stream=None,
             seed_shift: int = 1 << 40, cands=None, finalists: int = 8, log=None):
    """Return (best launch dict, table of (launch, kernel ms)) for ``systems``.

    Two stages: every candidate once, then the fastest ``finalists`` again
    with ``repeats`` timed runs each.  ``lnW``: optional per-system
    log-weights to time with.
    """
    scratch = [(d, L, N, W, lo, hi, seed + seed_shift) for (d, L, N, W, lo, hi, seed) in systems]
    first = []
    with m.Mucal(scratch, cuda_stream=cuda_stream) as mc:
        if lnW is not None:
            for i, w in enumerate(lnW):
                if w is not None:
                    mc.set_weights(i, w)
        it = 0
        seen = set()
        for cfg in (cands or with_threshold_modes(candidates())):
            try:
                mc.set_launch(**cfg)
            except m.MucalError:
                continue
            # shapes the library resolves to the same launch are timed once
            eff = tuple(sorted(mc.launch().items()))
            if eff in seen:
                continue
            seen.add(eff)
            try:
                ms, it = _time(mc, cfg, sweeps, 1, it)
            except m.MucalError:
                continue
            first.append((cfg, ms))
        first.sort(key=lambda x: x[1])
        table = []
        for cfg, _ in first[:finalists]:
            # each finalist also as a persistent launch (resident blocks that
            # pull the next block of walkers from a counter)
            for c in (cfg, dict(cfg, persistent=1)):
                try:
                    ms, it = _time(mc, c, sweeps, repeats, it)
                except m.MucalError:
                    continue
                table.append((c, ms))
                if log:
                    log(json.dumps({"launch": c, "kernel_ms": ms}))
    table.sort(key=lambda x: x[1])
    return table[0][0], table + first[finalists:]


def with_threshold_modes(cands):
    """Every group and field candidate also with thr_window = 0 (thresholds
    read from global memory when the table does not fit in shared memory;
    the default 1 keeps a window of rows per walker there instead), and at
    4 lanes or more with multi-commit rounds (which read the rows directly)."""
    out = []
    for c in cands:
        out.append(c)
        if c["kernel"] != m.MUCAL_KERNEL_THREAD:
            out.append(dict(c, thr_window=0))
            if c["lanes_per_walker"] >= 4:
                out.append(dict(c, thr_window=0, multi_commit=1))
    return out
