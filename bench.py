#!/usr/bin/env python3
"""Benchmark: attempted moves/s of the parallel multicanonical iteration on GB300.

One step = one iteration of the method (Sec. 2) over the whole workload:
every walker performs sweeps*N attempted jump moves with fixed weights
(walker-update kernel), the per-walker histograms are summed on the device
(Eq. 2), and the weights are updated by the recursion and redistributed as a
new threshold table.  Steps continue the same weight iteration from lnW = 0:
the W warm-up steps are its first iterations, the K timed steps the next ones.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1401_4076_gb300 import workloads  # noqa: E402

WORKLOADS = {
    "small2d": workloads.SMALL_2D,
    "medium2d": workloads.MEDIUM_2D,
    "large3d": workloads.LARGE_3D,
    "batched": workloads.batched_uneven(),
}
# one-system workloads timed briefly beside the headline
EXTRA_WORKLOADS = ("medium2d", "large3d")
METRIC = "attempted moves/s"

# Algorithmic integer work per attempted move, in thread-instruction
# equivalents, for the issue-slot roofline: one Philox4x32-10 block counted
# as 70 integer operations (ten rounds of two 32x32->64 multiplies, the xors
# with the key and the key bumps: 60-80 operations depending on how a
# wide multiply is counted; the middle is taken), the two multiply-high index
# maps (2), the reads of P[k] and Q[m] (2), the 2*2d occupancy bit tests
# (4d), the threshold compare (1) and the histogram increment (1):
# 84 in 2D, 88 in 3D.
PHILOX_OPS = 70


def alg_ops_per_attempt(d: int) -> int:
    return PHILOX_OPS + 2 + 2 + 4 * d + 1 + 1


# DRAM bytes (read + write) of one walker-update launch of a workload's
# default iteration, from the one-pass ncu capture summarised under profiles/,
# valid only for the launch shape and the kernel source it was taken with
# (sha256 prefix of walker_chain.cuh); any other shape or any change to the
# kernel makes the figure stale (null).  The persistent flag is not part of
# the shape here: when every block is resident at once (147 blocks of 28
# walkers on 152 SMs) the persistent launch runs the same blocks.
TRAFFIC_MEASURED = {
    # one full 1000-sweep launch (profiles/walker_update_field_2d-L64-N410-w4096.md)
    "2d-L64-N410-w4096": {"bytes": 34.239e6 + 802.815e6, "kernel_sha": "4f112a9b4d61e7f4",
                          "launch": {"kernel": 2, "lanes_per_walker": 8, "walkers_per_block": 28,
                                     "thr_window": 0, "multi_commit": 0}},
    # one full 200-sweep launch (profiles/walker_update_group_batched-27-systems-w16384.md)
    # (and the multi-commit shape the autotuner also picks there, by under 1 %)
    "batched-27-systems-w16384": [
        {"bytes": 704.779e9 + 300.284e9, "kernel_sha": "4f112a9b4d61e7f4",
         "launch": {"kernel": 1, "lanes_per_walker": 16, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 0}},
        {"bytes": 761.331e9 + 317.758e9, "kernel_sha": "4f112a9b4d61e7f4",
         "launch": {"kernel": 1, "lanes_per_walker": 8, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 1}},
    ],
    # a 5-sweep launch scaled by 40 to the workload's 200 sweeps (the list reads and
    # writes grow with the attempts; profiles/walker_update_group_3d-L32-N3277-w8192.md),
    # with multi-commit rounds and with one commit per round
    "3d-L32-N3277-w8192": [
        {"bytes": 40 * (18.5970e9 + 7.0710e9), "kernel_sha": "4f112a9b4d61e7f4",
         "launch": {"kernel": 1, "lanes_per_walker": 4, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 1}},
        {"bytes": 40 * (18.4596e9 + 7.0481e9), "kernel_sha": "4f112a9b4d61e7f4",
         "launch": {"kernel": 1, "lanes_per_walker": 4, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 0}},
    ],
}

# Executed instructions per attempted move of the walker-update kernel, from
# one ncu capture of a launch of the workload (smsp__inst_executed.sum x 32
# and smsp__thread_inst_executed.sum, divided by the launch's attempts), under
# the same validity rule as the traffic record: launch shape and kernel source.
INSTR_MEASURED = {
    # the full 1000-sweep launch of the traffic record
    "2d-L64-N410-w4096": {"warp_inst_per_attempt": 4.0031106e10 / 1.67936e9,
                          "thread_inst_per_attempt": 1.0419877e12 / 1.67936e9,
                          "kernel_sha": "4f112a9b4d61e7f4",
                          "launch": {"kernel": 2, "lanes_per_walker": 8, "thr_window": 0,
                                     "multi_commit": 0}},
    # 2-sweep launch, same shape as the traffic record (instructions per attempt do not
    # depend on the sweep count beyond the per-block set-up)
    "batched-27-systems-w16384": [
        {"warp_inst_per_attempt": 4.215209e9 / 72.3314e6,
         "thread_inst_per_attempt": 1.21995e11 / 72.3314e6,
         "kernel_sha": "4f112a9b4d61e7f4", "any_sweeps": True,
         "launch": {"kernel": 1, "lanes_per_walker": 16, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 0}},
        {"warp_inst_per_attempt": 3.788915e9 / 72.3314e6,
         "thread_inst_per_attempt": 1.0942e11 / 72.3314e6,
         "kernel_sha": "4f112a9b4d61e7f4", "any_sweeps": True,
         "launch": {"kernel": 1, "lanes_per_walker": 8, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 1}},
    ],
    "3d-L32-N3277-w8192": [
        {"warp_inst_per_attempt": 4.781667e9 / 134.2259e6,
         "thread_inst_per_attempt": 1.426715e11 / 134.2259e6,
         "kernel_sha": "4f112a9b4d61e7f4", "any_sweeps": True,
         "launch": {"kernel": 1, "lanes_per_walker": 4, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 1}},
        {"warp_inst_per_attempt": 2.974781e9 / 134.2259e6,
         "thread_inst_per_attempt": 8.90372e10 / 134.2259e6,
         "kernel_sha": "4f112a9b4d61e7f4", "any_sweeps": True,
         "launch": {"kernel": 1, "lanes_per_walker": 4, "bits_in_smem": 1, "thr_window": 0,
                    "multi_commit": 0}},
    ],
}

KERNEL_NAMES = {0: "walker_update_thread", 1: "walker_update_group", 2: "walker_update_field"}


def _kernel_sha() -> str:
    import hashlib
    # the walker-update kernels are compiled from walker_chain.cuh
    with open(os.path.join(ROOT, "paper_1401_4076_gb300", "csrc", "walker_chain.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _record_for(table: dict, workload: str, sweeps_default: bool, launch: dict):
    recs = table.get(workload)
    if recs is None:
        return None
    for rec in (recs if isinstance(recs, list) else [recs]):
        if not (sweeps_default or rec.get("any_sweeps")):
            continue
        # the launch keys a record names must match (records name the kernel,
        # the lanes per walker, the bitset staging, the threshold mode and the
        # rounds; the split into blocks does not change the per-attempt work
        # or access pattern)
        if any(launch.get(k) != v for k, v in rec["launch"].items()):
            continue
        if _kernel_sha() == rec["kernel_sha"]:
            return rec
    return None


def _measured_traffic(workload: str, sweeps_default: bool, launch: dict):
    rec = _record_for(TRAFFIC_MEASURED, workload, sweeps_default, launch)
    return None if rec is None else rec["bytes"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def shard_systems(systems, rank):
    """Walkers of rank r: every system keeps its walker count per rank, with
    walker seeds shifted past every walker of the lower ranks, so the ranks
    together run one multicanonical simulation with world x n_walkers
    walkers per system (weak scaling: fixed work per GPU)."""
    total = sum(s[3] for s in systems)
    out = []
    for (d, L, N, W, lo, hi, seed) in systems:
        out.append((d, L, N, W, lo, hi, seed + rank * total))
    return out


def allreduce_histograms(mc, n_sys, world, device):
    """Eq. 2 across processes: sum every system's histogram over the ranks
    (one int64 all-reduce per iteration) and hand the totals back, so that
    every rank computes the same next weights."""
    if world <= 1:
        return
    import torch
    import torch.distributed as dist
    Hs = [mc.histogram(s) for s in range(n_sys)]
    sizes = [h.size for h in Hs]
    t = torch.from_numpy(np.concatenate(Hs)).to(device)
    dist.all_reduce(t)
    tot = t.cpu().numpy()
    off = 0
    for s, n in enumerate(sizes):
        mc.set_histogram(s, tot[off:off + n])
        off += n


def cpu_oracle_rate(wl, budget_s: float, seed_offset: int = 0):
    """Attempted moves/s of the oracle (plain C, OpenMP over walkers) on a
    bounded sample of the workload: its first system(s), all walkers' seeds
    from the workload, lnW = 0, as many sweeps as fit the time budget."""
    from oracle import chain
    # calibrate on the largest-work system with a short run
    d, L, N, W, lo, hi, seed = max(wl.systems, key=lambda s: s[2] * s[3] * s[0])
    seed += seed_offset
    e_lo, e_hi = (-d * N, 0) if (lo == 0 and hi == 0) else (lo, hi)
    nw = min(W, max(chain.num_threads() * 4, 16))
    S, occ, E = chain.init_walkers(d, L, N, nw, seed)
    T = chain.thresholds(d, e_lo, e_hi, np.zeros(e_hi - e_lo + 1))
    cal = 1
    while True:
        t0 = time.perf_counter()
        chain.run_walkers(d, L, N, seed, 0, cal * N, e_lo, e_hi, T, S, occ, E)
        dt = time.perf_counter() - t0
        if dt > 0.25 or cal > (1 << 30):
            break
        cal *= 4
    sweeps = max(1, int(budget_s * cal / dt))
    t0 = time.perf_counter()
    chain.run_walkers(d, L, N, seed, 1, sweeps * N, e_lo, e_hi, T, S, occ, E)
    dt = time.perf_counter() - t0
    attempts = nw * sweeps * N
    sample = (f"system d={d} L={L} N={N}: {nw} of its {W} walkers x {sweeps} sweeps "
              f"({attempts} attempts), lnW=0, {dt:.1f} s")
    return attempts / dt, chain.num_threads(), sample


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    from oracle.build import build_oracle
    build_oracle()
    per_step = max(1.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, per_step * 0.2)
    rates = []
    samples = []
    cores = 1
    for _ in range(args.steps):
        r, cores, s = cpu_oracle_rate(wl, per_step)
        rates.append(r)
        samples.append(s)
    value = float(statistics.mean(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": _config(wl, args),
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                         "sample": samples[-1]},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(wl, args):
    return {"workload": wl.name, "systems": len(wl.systems),
            "walkers": sum(s[3] for s in wl.systems),
            "sweeps_per_iteration": args.sweeps or wl.sweeps,
            "attempts_per_step": (args.sweeps or wl.sweeps) * sum(s[2] * s[3] for s in wl.systems),
            "weights": "recursive update from lnW=0; timed steps are iterations P+W..P+W+K-1",
            "prerun_iterations": getattr(args, "prerun", 0),
            "l2": "flushed (512 MB write) before every timed step",
            "launch": getattr(args, "launch_desc", None),
            "cuda_graph": bool(getattr(args, "graph", False))}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mucal", "reference"], default="mucal")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batched",
                    help="the headline workload (default: the 27-system batch, the largest "
                         "workload on one GPU)")
    ap.add_argument("--sweeps", type=int, default=0, help="override sweeps per iteration")
    ap.add_argument("--walkers", type=int, default=0,
                    help="override the walker count of a one-system workload (the workload "
                         "name's -w suffix follows)")
    ap.add_argument("--kernel", type=int, default=-1)
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--wpb", type=int, default=0)
    ap.add_argument("--smem", type=int, default=-1)
    ap.add_argument("--thr-window", type=int, default=-1,
                    help="0: thresholds from global memory when the table does not fit in "
                         "shared memory, 1: per-walker row windows, 2: windows always")
    ap.add_argument("--multi-commit", type=int, default=-1,
                    help="1: several commits per round (group and field kernels, 4+ lanes), "
                         "0: one commit per round")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the launch-shape autotuner (run after the warm-up steps)")
    ap.add_argument("--tune-sweeps", type=int, default=20)
    ap.add_argument("--prerun", type=int, default=0,
                    help="untimed iterations of the recursion before the warm-up (to measure "
                         "a later stage of the weight iteration; 0 = start at lnW = 0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the learned-vs-plain convergence comparison (run after the timing)")
    ap.add_argument("--graph", action="store_true",
                    help="run every iteration's device work as one CUDA graph launch")
    ap.add_argument("--persistent", type=int, default=-1,
                    help="1: persistent walker-update launch, 0: one block per work item")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the short timings of the one-system workloads (2D L=64 and "
                         "3D L=32) reported beside the headline")
    ap.add_argument("--no-ceiling", action="store_true",
                    help="skip the latency ceiling (single-warp runs of every system)")
    ap.add_argument("--no-aux", action="store_true",
                    help="skip the timings of the analysis kernels (run after the timing)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]
    if args.walkers:
        if len(wl.systems) != 1 or args.walkers < 1:
            ap.error("--walkers needs a one-system workload and a count >= 1")
        import dataclasses
        import re
        d, L, N, _, lo, hi, seed = wl.systems[0]
        wl = dataclasses.replace(wl, name=re.sub(r"-w\d+$", f"-w{args.walkers}", wl.name),
                                 systems=((d, L, N, args.walkers, lo, hi, seed),))
    world, rank, local = _dist_setup()
    args.launch_desc = None

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        rc = run_reference(args, wl, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return rc

    import torch

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    # one explicit stream for the library and for torch's own work (the L2
    # flush): the timing events are recorded on the stream the kernels run on
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    systems = shard_systems(wl.systems, rank)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=device)

    res = measure(wl, args, systems, stream, device, world, flush, clocks_rank0=(rank == 0),
                  ceiling=not args.no_ceiling)
    line = {"metric": METRIC, "value": res["value"], "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": _config(wl, args), "roofline": res["roofline"],
            "clocks": res["clocks"], "gpu_launches": res["gpu_launches"],
            "acceptance": res["acceptance"]}

    if not args.no_e2e:
        line["e2e"] = e2e_measure(wl, args, systems, stream, device, world)
    if rank == 0 and world == 1 and not args.no_extra_workloads:
        extra = {}
        for name in EXTRA_WORKLOADS:
            if WORKLOADS[name].name == wl.name:
                continue
            xw = WORKLOADS[name]
            xargs = argparse.Namespace(**dict(vars(args), steps=5, warmup=3, sweeps=0, prerun=0,
                                              launch_desc=None))
            r = measure(xw, xargs, xw.systems, stream, device, 1, flush, clocks_rank0=False,
                        ceiling=not args.no_ceiling)
            extra[xw.name] = {"value": r["value"], "unit": "attempts/s",
                              "ms_per_step": r["ms_per_step"], "steps": 5, "warmup": 3,
                              "acceptance": r["acceptance"], "launch": xargs.launch_desc,
                              "attempts_per_step": xw.attempts_per_iteration(),
                              "roofline": r["roofline"]}
        line["workloads"] = extra
    if rank == 0 and world == 1 and not args.no_convergence:
        line["convergence_full_range"] = convergence_full_range(stream)
        line["convergence_half_window"] = convergence_measure(stream)
    if rank == 0 and world == 1 and not args.no_aux:
        line["aux_kernels"] = aux_measure(stream, device)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle.build import build_oracle
        build_oracle()
        r, cores, sample = cpu_oracle_rate(wl, args.cpu_budget)
        line["cpu_baseline"] = {"value": r, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                                "sample": sample}
        if not args.no_aux:
            line["cpu_baseline"]["aux_kernels"] = aux_oracle_rates()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _explicit_launch(args):
    return (args.kernel >= 0 or args.lanes or args.wpb or args.smem >= 0 or args.persistent >= 0
            or args.thr_window >= 0 or args.multi_commit >= 0)


def measure(wl, args, systems, stream, device, world, flush, clocks_rank0=True, ceiling=True):
    """The timed steps of one workload: W warm-up iterations of the weight
    recursion from lnW = 0, the launch-shape autotuner, then K timed
    iterations (walker update, histogram sums, histogram all-reduce across
    ranks, weight update and threshold upload), each bracketed by CUDA events
    on the library's stream after an L2 flush.  Returns the timing, the
    roofline of the walker-update kernel and (optionally) its latency ceiling."""
    import torch
    from paper_1401_4076_gb300 import mucal as m
    sweeps = args.sweeps or wl.sweeps
    attempts_per_step = sweeps * sum(s[2] * s[3] for s in systems)
    mc = m.Mucal(systems, cuda_stream=stream.cuda_stream)
    if _explicit_launch(args):
        cur = mc.launch()
        cfg = dict(kernel=args.kernel if args.kernel >= 0 else cur["kernel"],
                   lanes_per_walker=args.lanes or cur["lanes_per_walker"],
                   walkers_per_block=args.wpb or cur["walkers_per_block"],
                   bits_in_smem=args.smem if args.smem >= 0 else cur["bits_in_smem"],
                   persistent=args.persistent if args.persistent >= 0 else cur["persistent"],
                   thr_window=args.thr_window if args.thr_window >= 0 else 1,
                   multi_commit=args.multi_commit if args.multi_commit >= 0 else 0)
        mc.set_launch(**cfg)
    if args.graph:
        mc.set_graph_mode(True)
    args.launch_desc = mc.launch()
    n_sys = len(systems)

    def step(it):
        mc.run_iteration(sweeps, it)
        allreduce_histograms(mc, n_sys, world, device)
        for s in range(n_sys):
            mc.update_weights(s, m.MUCAL_SCHEME_RECURSIVE)

    for it in range(args.prerun):
        step(it)
    for it in range(args.prerun, args.prerun + args.warmup):
        step(it)
    torch.cuda.synchronize(device)
    if not args.no_autotune and not _explicit_launch(args):
        from paper_1401_4076_gb300.autotune import autotune
        lnWs = [mc.weights(s) for s in range(n_sys)]
        best, table = autotune(systems, lnW=lnWs, sweeps=args.tune_sweeps, repeats=5,
                               cuda_stream=stream.cuda_stream)
        mc.set_launch(**best)
        args.launch_desc = mc.launch()
        for cfg, ms in table[:5]:
            print(json.dumps({"workload": wl.name, "autotune": cfg, "kernel_ms": ms}),
                  file=sys.stderr)
    torch.cuda.synchronize(device)
    _barrier(world)
    torch.cuda.synchronize(device)

    clocks = ClockSampler(device.index or 0) if clocks_rank0 else None
    if clocks:
        clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    accs = []
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step(args.prerun + args.warmup + i)
        ends[i].record(stream)
        st = [mc.stats(s) for s in range(n_sys)]
        kernel_ms.append(st[0]["kernel_ms"])
        accs.append(sum(x["accepts"] for x in st) / max(1, sum(x["attempts"] for x in st)))
    torch.cuda.synchronize(device)
    _barrier(world)
    torch.cuda.synchronize(device)
    clk = clocks.stop() if clocks else None
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    step_ms = _max_over_ranks(step_ms, world, device)
    value = attempts_per_step * args.steps * world / (step_ms / 1000.0)

    # dominant kernel (walker update): algorithmic integer ops per launch / its
    # average duration (CUDA events on the library's stream around the launch)
    d_max = max(s[0] for s in systems)
    ops_launch = sum(alg_ops_per_attempt(s[0]) * s[2] * s[3] * sweeps for s in systems)
    k_ms = statistics.mean(kernel_ms)
    peaks, peak_kind = _peaks()
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    f_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_ops = sm_count * 128 * f_mhz * 1e6          # thread-instructions/s
    achieved = ops_launch / (k_ms / 1000.0)
    kernel_rate = attempts_per_step / (k_ms / 1000.0)
    blocks_per_sm, _ = mc.occupancy()
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s", "frac": achieved / peak_ops,
                "traffic": _measured_traffic(wl.name, sweeps == wl.sweeps, args.launch_desc),
                "peak_source": f"{sm_count} SMs x 128 lanes x {f_mhz} MHz ({peak_kind} max clock)",
                "kernel": KERNEL_NAMES.get(args.launch_desc.get("kernel"), "walker_update"),
                "kernel_ms": k_ms,
                "kernel_attempts_per_s": kernel_rate,
                "alg_ops_per_attempt": alg_ops_per_attempt(d_max),
                "alg_ops_basis": "Philox 70 + index maps 2 + list reads 2 + bit tests 4d + "
                                 "threshold 1 + histogram 1",
                "chains_per_sm": sum(s[3] for s in systems) / sm_count,
                "resident_blocks_per_sm": blocks_per_sm}
    rec = _record_for(INSTR_MEASURED, wl.name, sweeps == wl.sweeps, args.launch_desc)
    if rec is not None:
        # issue slots: 4 warp instructions per SM and clock
        roofline["issue"] = {"warp_inst_per_attempt": rec["warp_inst_per_attempt"],
                             "thread_inst_per_attempt": rec["thread_inst_per_attempt"],
                             "frac": kernel_rate * rec["warp_inst_per_attempt"] / 32.0
                             / (sm_count * 4 * f_mhz * 1e6)}
    lnWs = [mc.weights(s) for s in range(n_sys)]
    mc.close()
    if ceiling:
        try:
            roofline["latency_ceiling"] = latency_ceiling(systems, lnWs, args.launch_desc, sweeps,
                                                          stream, blocks_per_sm, sm_count,
                                                          kernel_rate)
        except Exception as exc:   # reported, never fatal for the benchmark line
            roofline["latency_ceiling"] = {"error": repr(exc)[:200]}
    # launches inside the timed region: per step one walker update and one
    # histogram-reduce launch per system (the clears are driver memsets)
    return {"value": value, "ms_per_step": step_ms / args.steps, "roofline": roofline,
            "clocks": clk, "gpu_launches": args.steps * (1 + n_sys),
            "acceptance": statistics.mean(accs)}


def latency_ceiling(systems, lnWs, launch, sweeps, stream, blocks_per_sm, sm_count, kernel_rate):
    """What the launch's parallelism allows if its chains never waited for one
    another: every system's walkers run alone, one warp (32 / lanes walkers)
    on an otherwise idle GPU, with the weights of the timed steps and the
    launch's kernel and lanes; that warp's attempted moves per second is the
    inverse of its critical path per attempt.  The ceiling is the number of
    warps resident at once (occupancy of the launch shape, at most the
    launch's warps) times the attempt-weighted mean single-warp rate."""
    from paper_1401_4076_gb300 import mucal as m
    G = max(1, launch["lanes_per_walker"])
    per_warp = 32 // G
    rates = []
    work = []
    for i, (d, L, N, W, lo, hi, seed) in enumerate(systems):
        desc = (d, L, N, per_warp, lo, hi, seed + (1 << 41))
        sw = max(1, int(4e5 // (per_warp * N)))
        with m.Mucal([desc], cuda_stream=stream.cuda_stream) as mc:
            mc.set_weights(0, lnWs[i])
            shape = dict(launch, walkers_per_block=per_warp, persistent=0)
            try:
                mc.set_launch(**shape)
            except m.MucalError:
                mc.set_launch(**dict(shape, bits_in_smem=0))
            mc.run_iteration(sw, 0)
            mc.run_iteration(sw, 1)
            ms = mc.stats(0)["kernel_ms"]
        rates.append(per_warp * sw * N / (ms / 1000.0))
        work.append(W * sweeps * N)
    t_mean = sum(a / r for a, r in zip(work, rates)) / sum(work)   # s per attempt per warp
    warps_per_block = max(1, launch["walkers_per_block"] * G // 32)
    launch_warps = sum(-(-s[3] // launch["walkers_per_block"]) for s in systems) * warps_per_block
    resident = min(launch_warps, blocks_per_sm * warps_per_block * sm_count)
    ceil = resident / t_mean
    return {"value": ceil, "unit": "attempts/s", "frac": kernel_rate / ceil,
            "resident_warps": resident, "launch_warps": launch_warps,
            "single_warp_attempts_per_s": 1.0 / t_mean,
            "basis": "resident warps x attempt-weighted single-warp rate (each system alone, "
                     "one warp, weights of the timed steps)"}


AUX_SYSTEM = (2, 64, 410, 4096, 0, 0, 0)   # the 2D L=64, N=410, 4096-walker system


def _events_ms(stream, fn, reps):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def aux_measure(stream, device):
    """Device times of the analysis kernels on the 2D L=64, N=410 system with
    4096 walkers, each against the HBM roofline of its algorithmic bytes:
    droplet labelling (reads every walker's particle list and bitset, writes
    V_D), replica exchange on an 8-copy ladder at equal temperatures (every
    proposal accepted: both configurations read and written), and the cost of
    the tunnelling flavour of the walker kernel."""
    from paper_1401_4076_gb300 import mucal as m
    out = {}
    peaks, kind = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    d, L, N, W, _, _, _ = AUX_SYSTEM
    V = L ** d
    try:
        with m.Mucal([AUX_SYSTEM], cuda_stream=stream.cuda_stream) as mc:
            mc.set_weights(0, -1.2 * np.arange(d * N + 1, dtype=np.float64))
            mc.run_iteration(20, 0)                 # bonds favoured: droplets form
            ms = _events_ms(stream, mc.measure_droplets, 20)
            bytes_ = W * (N * 2 + V // 8 + 4 + 4)
            vd = mc.largest_droplets(0)
            out["droplet_labelling"] = {
                "ms_per_measurement": ms, "walkers_per_s": W / (ms / 1e3),
                "mean_V_D": float(vd.mean()),
                "roofline": {"bound": "hbm", "alg_bytes": bytes_,
                             "achieved": bytes_ / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": bytes_ / (ms / 1e3) / 1e9 / hbm,
                             "peak_source": f"{kind} hbm_gbs"}}
            mc.run_iteration(100, 1)
            k_plain = mc.stats(0)["kernel_ms"]
            mc.set_tunnel_window(0, 0, 0)
            mc.run_iteration(100, 2)
            k_tun = mc.stats(0)["kernel_ms"]
            out["tunnelling_flavour"] = {"walker_kernel_ms_plain": k_plain,
                                         "walker_kernel_ms_tunnel": k_tun,
                                         "cost": k_tun / k_plain - 1.0,
                                         "sweeps": 100}
    except Exception as exc:
        out["droplet_error"] = repr(exc)[:200]
    try:
        # the same labelling on the 3D L=32 system: 8192 walkers, 87 MB per measurement
        d3, L3, N3, W3, _, _, _ = workloads.LARGE_3D.systems[0]
        V3 = L3 ** d3
        with m.Mucal(workloads.LARGE_3D.systems, cuda_stream=stream.cuda_stream) as mc:
            mc.set_weights(0, -1.2 * np.arange(d3 * N3 + 1, dtype=np.float64))
            mc.run_iteration(5, 0)
            ms = _events_ms(stream, mc.measure_droplets, 5)
            bytes_ = W3 * (N3 * 2 + V3 // 8 + 4 + 4)
            vd = mc.largest_droplets(0)
            out["droplet_labelling_3d"] = {
                "system": "3D L=32, N=3277, 8192 walkers",
                "ms_per_measurement": ms, "walkers_per_s": W3 / (ms / 1e3),
                "mean_V_D": float(vd.mean()),
                "roofline": {"bound": "hbm", "alg_bytes": bytes_,
                             "achieved": bytes_ / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": bytes_ / (ms / 1e3) / 1e9 / hbm,
                             "peak_source": f"{kind} hbm_gbs"}}
    except Exception as exc:
        out["droplet_3d_error"] = repr(exc)[:200]
    try:
        K = 8
        ladder = [(d, L, N, W, 0, 0, 10 ** 7 + k * W) for k in range(K)]
        with m.Mucal(ladder, cuda_stream=stream.cuda_stream) as mc:
            betas = [1.0] * K
            r = [0]

            def ex():
                mc.replica_exchange(betas, r[0], 0)
                r[0] += 1
            ms = _events_ms(stream, ex, 20)
            pairs = K // 2
            bytes_ = pairs * W * 2 * 2 * (V * 2 + V // 8 + 4)
            out["replica_exchange"] = {
                "ms_per_call": ms, "ladder": f"{K} copies, parity 0 ({pairs} pairs), all accepted",
                "note": "each call also uploads the threshold rows and reads back the counts",
                "roofline": {"bound": "hbm", "alg_bytes": bytes_,
                             "achieved": bytes_ / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": bytes_ / (ms / 1e3) / 1e9 / hbm,
                             "peak_source": f"{kind} hbm_gbs"}}
    except Exception as exc:
        out["exchange_error"] = repr(exc)[:200]
    try:
        from paper_1401_4076_gb300 import workloads as wls
        params = wls.mlp_initial_params(0)
        X, t = wls.mlp_test_batch(8192, 1)
        res = {}
        for name, tc in (("tcgen05", True), ("mma_sync", False)):
            with m.Mlp(params, cuda_stream=stream.cuda_stream) as net:
                net.use_tcgen05(tc)
                net.train(X, t, steps=20, lr=1e-3)
                t0 = time.perf_counter()
                net.train(X, t, steps=200, lr=1e-3)
                step_ms = (time.perf_counter() - t0) / 200 * 1e3
                net.forward(X)
                t0 = time.perf_counter()
                for _ in range(20):
                    net.forward(X)
                fwd_ms = (time.perf_counter() - t0) / 20 * 1e3
            # flops of the three 128x128 contractions per row (forward with
            # hi + lo: 2 x 2 H^2; backward: dH1 and dW2: 2 x 2 H^2)
            flops = 8192 * 8 * 128 * 128
            res[name] = {"train_step_ms": step_ms, "forward_ms_with_copies": fwd_ms,
                         "train_tflops_effective": flops / (step_ms / 1e3) / 1e12}
        out["seeding_network"] = dict(res, batch=8192,
                                      note="train step = gradient kernels + Adam, host loop; "
                                           "forward includes the host-device copies")
    except Exception as exc:
        out["mlp_error"] = repr(exc)[:200]
    try:
        rng = np.random.default_rng(0)
        H = rng.integers(1, 10 ** 6, d * N + 1)
        lnW = np.cumsum(rng.normal(size=d * N + 1))
        betas = np.linspace(0.1, 3.0, 1000)
        t0 = time.perf_counter()
        m.mucal_reweight(H, lnW, -d * N, betas)
        out["reweighting"] = {"betas": 1000, "bins": d * N + 1,
                              "host_ms": (time.perf_counter() - t0) * 1e3}
    except Exception as exc:
        out["reweight_error"] = repr(exc)[:200]
    return out


def aux_oracle_rates():
    """The oracle beside the analysis kernels: breadth-first largest droplet
    per walker (one thread) on the oracle's own placements of the same
    system, the replica exchange on a 64-walker 8-copy ladder, and the
    reweighting of 1000 temperatures."""
    from oracle import chain, muca
    out = {}
    d, L, N, W, _, _, seed = AUX_SYSTEM
    nw = 64
    S, occ, E = chain.init_walkers(d, L, N, nw, seed)
    t0 = time.perf_counter()
    for w in range(nw):
        chain.largest_droplet(d, L, occ[w])
    dt = time.perf_counter() - t0
    out["droplet_labelling"] = {"walkers_per_s": nw / dt, "cores": 1,
                                "sample": f"{nw} random placements of 64x64, N=410"}
    K = 8
    V = L ** d
    seeds = np.array([10 ** 7 + k * W for k in range(K)], dtype=np.uint64)
    SS = np.zeros((K, nw, V), np.int32)
    OO = np.zeros((K, nw, V), np.uint8)
    EE = np.zeros((K, nw), np.int64)
    for k in range(K):
        SS[k], OO[k], EE[k] = chain.init_walkers(d, L, N, nw, int(seeds[k]))
    t0 = time.perf_counter()
    for r in range(5):
        chain.replica_exchange([1.0] * K, seeds, r, 0, SS, OO, EE)
    dt = (time.perf_counter() - t0) / 5
    out["replica_exchange"] = {"ms_per_call": dt * 1e3, "cores": 1,
                               "sample": f"{K} copies x {nw} walkers (the GPU line: x 4096)"}
    rng = np.random.default_rng(0)
    H = rng.integers(1, 10 ** 6, d * N + 1)
    lnW = np.cumsum(rng.normal(size=d * N + 1))
    t0 = time.perf_counter()
    for b in np.linspace(0.1, 3.0, 100):
        muca.reweight_moments(lnW, H, -d * N, b)
    out["reweighting"] = {"ms_per_1000_betas": (time.perf_counter() - t0) * 1e4, "cores": 1,
                          "sample": "100 betas, scaled to 1000"}
    return out


def convergence_measure(stream):
    """Iterations and wall time to a flat histogram (min/max >= 0.5), plain
    start lnW = 0 with the recursion against the learned seed, on 2D L=64,
    N=410, 4096 walkers, 50 sweeps per iteration, window [-dN/2, 0].  The
    network is trained on the GPU first on small lattices run to flatness by
    the method itself (its time is reported separately)."""
    try:
        from paper_1401_4076_gb300 import seeding as sd
        t0 = time.perf_counter()
        small = sd.small_training_systems(0.5)
        res = sd.iterate_to_flat(small, sweeps=100, max_iter=200, final_sweeps=1000,
                                 cuda_stream=stream.cuda_stream)
        X, t = sd.training_set([r for r in res if r.converged])
        net, loss = sd.train(X, t, steps=20000, lr=1e-3, cuda_stream=stream.cuda_stream)
        prep = time.perf_counter() - t0
        d, L, N, W = 2, 64, 410, 4096
        lo, hi = sd.window_fraction(d, N, 0.5)
        plain, seeded, _ = sd.compare_plain_and_seeded(net, (d, L, N, W, lo, hi, 123456), 50, 300,
                                                       cuda_stream=stream.cuda_stream)
        net.close()
        return {"system": "2D L=64 N=410, 4096 walkers, window [-410, 0], 50 sweeps/iteration",
                "goal": "min/max H >= 0.5",
                "plain": {"iterations": plain.iterations, "wall_s": round(plain.wall_s, 3),
                          "converged": plain.converged},
                "learned": {"iterations": seeded.iterations, "wall_s": round(seeded.wall_s, 3),
                            "converged": seeded.converged},
                "training_s": round(prep, 3), "training_rows": int(len(t))}
    except Exception as exc:  # reported, never fatal for the benchmark line
        return {"error": repr(exc)[:200]}


def convergence_full_range(stream, seeds=(0, 1)):
    """Iterations and wall time to a flat histogram over the whole sampled
    energy range of 2D L=64, N=410 with 4096 walkers (the gas at E = 0 down
    to the compact droplet at E = -779): the plain start lnW = 0 against the
    learned seed, both with the two-stage iteration (simple update with the
    edge continuation; 1000-sweep iterations until the sampled range is
    stable, or a relaxation with the seed held fixed; then 4000 measured
    sweeps after 1000 discarded ones per iteration).  The network is first
    trained on small lattices the method itself ran to flatness over their
    whole ranges (its time is reported separately)."""
    try:
        from paper_1401_4076_gb300 import mucal as m
        from paper_1401_4076_gb300 import seeding as sd
        from paper_1401_4076_gb300.iterate import iterate_to_flat
        scheme = m.MUCAL_SCHEME_SIMPLE | m.MUCAL_SCHEME_EXTRAPOLATE
        t0 = time.perf_counter()
        small = sd.small_training_systems(1.0)
        res = iterate_to_flat(small, sweeps=100, max_iter=300, final_sweeps=1000, scheme=scheme,
                              cuda_stream=stream.cuda_stream)
        X, t = sd.training_set([r for r in res if r.converged])
        net, loss = sd.train(X, t, steps=20000, lr=1e-3, cuda_stream=stream.cuda_stream)
        prep = time.perf_counter() - t0
        d, L, N, W = 2, 64, 410, 4096
        runs = {"plain": [], "learned": []}
        for k in seeds:
            desc = (d, L, N, W, 0, 0, 7 * 10 ** 6 + k * W)
            plain, seeded, _ = sd.compare_staged(net, desc, max_iter=150, target=(-778, 0),
                                                 cuda_stream=stream.cuda_stream)
            for key, r in (("plain", plain), ("learned", seeded)):
                runs[key].append({"iterations": r.iterations, "stage1": r.range_iterations,
                                  "wall_s": round(r.wall_s, 3), "converged": r.converged,
                                  "flatness": round(float(r.flatness[-1]), 4),
                                  "sampled_range": list(r.span),
                                  "tunnel_events_stage2": r.tunnel_events})
        net.close()
        out = {"system": "2D L=64 N=410, 4096 walkers, window [-820, 0], flatness over "
                         "[-778, 0] (the compact droplet at -779 to the gas at 0)",
               "goal": "min/max H >= 0.5",
               "method": "stage 1: 1000-sweep iterations, simple update + edge continuation, "
                         "until the sampled range is stable for 5 (plain) / seed held fixed "
                         "(learned); stage 2: 1000 discarded + 4000 measured sweeps per iteration",
               "training_s": round(prep, 3), "training_rows": int(len(t)),
               "training_systems_converged": int(sum(r.converged for r in res))}
        for key, rs in runs.items():
            ok = [r for r in rs if r["converged"]]
            out[key] = {"runs": rs, "converged": f"{len(ok)}/{len(rs)}",
                        "mean_iterations": float(np.mean([r["iterations"] for r in rs])),
                        "mean_wall_s": float(np.mean([r["wall_s"] for r in rs]))}
        return out
    except Exception as exc:  # reported, never fatal for the benchmark line
        return {"error": repr(exc)[:200]}


def e2e_measure(wl, args, systems, stream, device, world):
    """The same metric end to end through the public API from host buffers: a
    fresh context (initial placement), then K iterations each uploading the new
    threshold table and reading the histogram back to the host."""
    import torch
    from paper_1401_4076_gb300 import mucal as m
    sweeps = args.sweeps or wl.sweeps
    attempts = sweeps * sum(s[2] * s[3] for s in systems) * args.steps
    torch.cuda.synchronize(device)
    _barrier(world)
    t0 = time.perf_counter()
    mc = m.Mucal(systems, cuda_stream=stream.cuda_stream)
    if args.launch_desc:
        mc.set_launch(**args.launch_desc)
    if args.graph:
        mc.set_graph_mode(True)
    h2d = d2h = 0
    for it in range(args.steps):
        mc.run_iteration(sweeps, it)
        allreduce_histograms(mc, len(systems), world, device)
        for s in range(len(systems)):
            H = mc.histogram(s)
            lnW, _ = mc.update_weights(s, m.MUCAL_SCHEME_RECURSIVE)
            i = mc.info[s]
            d2h += H.nbytes
            h2d += i["n_bins"] * i["width"] * 4
    torch.cuda.synchronize(device)
    dt = _max_over_ranks(time.perf_counter() - t0, world, device)
    mc.close()
    return {"value": attempts * world / dt, "unit": "attempts/s",
            "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
            "includes": "context creation + initial placement, K iterations with weight updates"}


if __name__ == "__main__":
    sys.exit(main())
