"""The iteration of Sec. 2 run to flatness through the library.

Every step runs in libmucal (walker update and histogram sum on the GPU,
float64 weight update and threshold build in the library's host code); this
module only loops over iterations, tracks the flatness the library reports
and collects results.  Also a command-line driver for convergence runs:

    python -m paper_1401_4076_gb300.iterate --system d:L:N:walkers \
        [--window lo:hi] [--target lo:hi] --sweeps S --max-iter K
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import mucal as m


def ln_binomial(V: int, N: int) -> float:
    return math.lgamma(V + 1) - math.lgamma(N + 1) - math.lgamma(V - N + 1)


def ln_omega_estimate(lnW: np.ndarray, H: np.ndarray, V: int, N: int) -> np.ndarray:
    """ln Omega(E) = ln H(E) - lnW(E) on visited bins (W = 1/Omega makes H flat,
    Sec. 2), shifted so that the visited bins carry all C(V, N) states; NaN
    where H = 0 (computed by the library)."""
    return m.mucal_ln_omega(H, lnW, V, N)


@dataclass
class RunResult:
    desc: tuple
    iterations: int
    flatness: list
    converged: bool
    wall_s: float
    lnW: np.ndarray
    H: np.ndarray
    attempts: int = 0
    extra: dict = field(default_factory=dict)


def ln_omega_multi(history, V: int, N: int) -> np.ndarray:
    """ln Omega(E) from several iterations' histograms and the weights they
    were sampled with (the multi-histogram combination of the library),
    shifted so that the visited bins carry all C(V, N) states."""
    H = np.stack([h for h, _ in history])
    W = np.stack([w for _, w in history])
    lo, _ = m.mucal_multi_histogram(H, W)
    return m.mucal_ln_omega_normalise(lo, V, N)


def iterate_to_flat(systems, sweeps: int, max_iter: int, targets=None, lnW0=None, goal=0.5,
                    scheme=m.MUCAL_SCHEME_RECURSIVE, cuda_stream=None, launch=None,
                    final_sweeps: int = 0, relax_iters: int = 0, relax_tol: float = 0.0,
                    history: int = 0, sweeps_growth: int = 1, stall: int = 10):
    """Run the weight iteration of Sec. 2 for several systems in one context
    (one launch per iteration) until each reaches flatness >= goal inside its
    target window (t_lo, t_hi) or max_iter iterations.  A system that has
    converged keeps running with frozen weights (its histogram then serves the
    ln Omega estimate).  Returns one RunResult per system.

    relax_iters: iterations run with the starting weights held fixed before
    the first update (their histograms are discarded).  Walkers start from
    random placements, which are equilibrium states of lnW = 0 only; the
    update of Sec. 2 assumes equilibrium runs, so a start from other weights
    first lets the walkers relax to them.  These iterations count towards
    the reported iterations and wall time.  With relax_tol > 0, relax_iters is
    a cap and the relaxation of a system ends early once the mean energy of
    its histogram moves by less than relax_tol times the window width from
    one iteration to the next.

    history: keep the histograms of the last `history` updating iterations of
    each system with the weights they were sampled with, in
    RunResult.extra["history"] (for ``ln_omega_multi``).

    sweeps_growth > 1: the sweeps per iteration double whenever no system's
    flatness has improved by more than 0.02 over its best for `stall`
    iterations, up to sweeps_growth times the starting value (more
    statistics per histogram once the weights are close; the systems of one
    context share one launch and therefore one sweep count).
    """
    n = len(systems)
    t0 = time.perf_counter()
    with m.Mucal(systems, cuda_stream=cuda_stream) as mc:
        if launch:
            mc.set_launch(**launch)
        for i in range(n):
            if lnW0 is not None and lnW0[i] is not None:
                mc.set_weights(i, lnW0[i])
            if targets is not None and targets[i] is not None:
                mc.set_target_window(i, *targets[i])
        done = [False] * n
        iters = [0] * n
        flat = [[] for _ in range(n)]
        walls = [0.0] * n
        attempts = [0] * n
        Hs = [None] * n
        relaxing = [relax_iters > 0] * n
        relaxed = [0] * n
        last_mean = [None] * n
        hist_keep = [[] for _ in range(n)]
        sw0 = sweeps
        best = [-1.0] * n
        since = 0
        sweeps_used = []
        for it in range(max_iter):
            mc.run_iteration(sweeps, it)
            sweeps_used.append(sweeps)
            for i in range(n):
                if done[i]:
                    continue
                iters[i] = it + 1
                attempts[i] += sweeps * systems[i][2] * systems[i][3]
                if relaxing[i]:
                    flat[i].append(float("nan"))
                    relaxed[i] += 1
                    stop = relaxed[i] >= relax_iters
                    if not stop and relax_tol > 0:
                        H = mc.histogram(i).astype(np.float64)
                        mean = float((H * np.arange(len(H))).sum() / max(H.sum(), 1.0))
                        if last_mean[i] is not None and abs(mean - last_mean[i]) < relax_tol * len(H):
                            stop = True
                        last_mean[i] = mean
                    if stop:
                        relaxing[i] = False
                    continue
                H = mc.histogram(i)
                if history:
                    hist_keep[i].append((H, mc.weights(i)))
                    del hist_keep[i][:-history]
                lnW, f = mc.update_weights(i, scheme)
                flat[i].append(f)
                Hs[i] = H
                if f >= goal:
                    done[i] = True
                    walls[i] = time.perf_counter() - t0
            if all(done):
                break
            if sweeps_growth > 1:
                improved = False
                for i in range(n):
                    if not done[i] and flat[i] and flat[i][-1] == flat[i][-1] and flat[i][-1] > best[i] + 0.02:
                        best[i] = flat[i][-1]
                        improved = True
                since = 0 if improved else since + 1
                if since >= stall and sweeps < sw0 * sweeps_growth:
                    sweeps *= 2
                    since = 0
                    best = [-1.0] * n
        for i in range(n):
            if not done[i]:
                walls[i] = time.perf_counter() - t0
        results = []
        final_H = [None] * n
        lnWs = [mc.weights(i) for i in range(n)]
        if final_sweeps:
            # one more iteration with the final weights for the ln Omega estimate
            for i in range(n):
                mc.set_weights(i, lnWs[i])
            mc.run_iteration(final_sweeps, max_iter + 1)
            for i in range(n):
                final_H[i] = mc.histogram(i)
        for i in range(n):
            extra = {"history": hist_keep[i]} if history else {}
            extra["sweeps"] = sweeps_used[:iters[i]]
            results.append(RunResult(tuple(systems[i]), iters[i], flat[i], done[i], walls[i],
                                     lnWs[i], final_H[i] if final_sweeps else Hs[i],
                                     attempts[i], extra))
    return results




@dataclass
class StagedResult:
    desc: tuple
    converged: bool
    iterations: int             # updating iterations of both stages (relaxation counted too)
    range_iterations: int       # stage 1 (or relaxation after a seed)
    wall_s: float
    flatness: list
    lnW: np.ndarray
    span: tuple                 # sampled energy range when stage 2 began
    tunnel_events: int          # end-to-end travels during stage 2 (Sec. 4) between the
                                # target's ends, else those of the sampled range
    sweeps: int                 # attempted sweeps of all iterations, discards included


def iterate_staged(desc, lnW0=None, range_sweeps: int = 1000, sweeps: int = 4000,
                   discard: int = 1000, max_iter: int = 200, stable: int = 5, goal: float = 0.5,
                   target=None, scheme=m.MUCAL_SCHEME_SIMPLE | m.MUCAL_SCHEME_EXTRAPOLATE,
                   relax_max: int = 10, cuda_stream=None, launch=None,
                   seed_range_stage: bool = False, progress=None) -> StagedResult:
    """The iteration of Sec. 2 in two stages for one system.

    Stage 1 (from lnW = 0): short iterations of `range_sweeps` with the simple
    update and the edge continuation, until the sampled energy range has not
    changed for `stable` iterations.  With a starting lnW0 (a learned seed)
    stage 1 is replaced by relaxation: iterations of `range_sweeps` with the
    seed held fixed inside the sampled range and continued at the sampled
    range's edges as the edge continuation does (so that the walkers reach
    energies where the seed is too steep), until the sampled range has not
    changed for `stable` iterations (at most `relax_max`); random placements
    are equilibrium states of lnW = 0 only; with seed_range_stage the
    relaxation is followed by stage 1 itself, started from the relaxed seed.
    Stage 2: iterations of `sweeps` measured sweeps, each after a
    discarded run of `discard` sweeps (Sec. 2 asks for equilibrium runs with
    fixed weights: the discard lets the walkers follow the last update),
    updated with `scheme`, until the flatness over the target window (default:
    the sampled range) reaches `goal`.  Tunnelling events over the sampled
    range (Sec. 4's criterion) are counted during stage 2.  `progress`, if
    given, is called after every stage-2 iteration with a dict (iteration,
    flatness, tunnelling events so far, wall time), so that a run cut short
    still leaves its trajectory."""
    d, L, N, W, lo, hi, seed = desc
    t0 = time.perf_counter()
    it_no = 0
    total_sweeps = 0
    flat = []
    with m.Mucal([desc], cuda_stream=cuda_stream) as mc:
        if launch:
            mc.set_launch(**launch)
        if lnW0 is not None:
            mc.set_weights(0, lnW0)
        if target is not None:
            mc.set_target_window(0, *target)
        e_lo = mc.info[0]["e_lo"]
        nb = mc.info[0]["n_bins"]
        span, same, n1 = None, 0, 0
        cap1 = max_iter if lnW0 is None else relax_max
        while same < stable and n1 < cap1:
            sw = range_sweeps
            mc.run_iteration(sw, it_no)
            it_no += 1
            n1 += 1
            total_sweeps += sw
            H = mc.histogram(0)
            vis = np.nonzero(H > 0)[0]
            sp = (int(vis.min()), int(vis.max()))
            if span is not None:
                sp = (min(sp[0], span[0]), max(sp[1], span[1]))
            same = same + 1 if sp == span else 0
            span = sp
            if lnW0 is None:
                _, f = mc.update_weights(0, scheme)
                flat.append(f)
            else:
                # the seed inside the sampled range, continued beyond it
                st = m.WeightState(nb, lnW0)
                st.visited[sp[0]:sp[1] + 1] = 1
                m.mucal_weight_update(st, np.zeros(nb, dtype=np.int64),
                                      m.MUCAL_SCHEME_SIMPLE | m.MUCAL_SCHEME_EXTRAPOLATE)
                mc.set_weights(0, st.lnW)
                if target is not None:
                    mc.set_target_window(0, *target)
                flat.append(float("nan"))
        if lnW0 is not None and seed_range_stage:
            # stage 1 from the relaxed seed: the updates correct where the seed is wrong
            mc.set_weights(0, mc.weights(0))
            if target is not None:
                mc.set_target_window(0, *target)
            same = 0
            k1 = 0
            while same < stable and n1 + k1 < max_iter:
                mc.run_iteration(range_sweeps, it_no)
                it_no += 1
                k1 += 1
                total_sweeps += range_sweeps
                H = mc.histogram(0)
                vis = np.nonzero(H > 0)[0]
                sp = (min(int(vis.min()), span[0]), max(int(vis.max()), span[1]))
                same = same + 1 if sp == span else 0
                span = sp
                _, f = mc.update_weights(0, scheme)
                flat.append(f)
            n1 += k1
        lnW = mc.weights(0)
        # stage 2 starts with a fresh recursion memory (the stage-1 histograms
        # come from walkers far from equilibrium)
        mc.set_weights(0, lnW)
        if target is not None:
            mc.set_target_window(0, *target)
        # tunnelling events between the target's ends (else the sampled range's)
        mc.set_tunnel_window(0, *(target if target is not None else
                                  (e_lo + span[0], e_lo + span[1])))
        converged = False
        n2 = 0
        while n1 + n2 < max_iter:
            if discard:
                mc.run_iteration(discard, it_no)
                it_no += 1
                total_sweeps += discard
            mc.run_iteration(sweeps, it_no)
            it_no += 1
            n2 += 1
            total_sweeps += sweeps
            _, f = mc.update_weights(0, scheme)
            flat.append(f)
            if progress is not None:
                progress({"iteration": n1 + n2, "stage2_iteration": n2, "flatness": f,
                          "tunnel_events_stage2": int(mc.tunnel_counts(0)[0]),
                          "wall_s": round(time.perf_counter() - t0, 3)})
            if f >= goal:
                converged = True
                break
        tun = mc.tunnel_counts(0)[0]
        lnW = mc.weights(0)
    return StagedResult(tuple(desc), converged, n1 + n2, n1, time.perf_counter() - t0, flat, lnW,
                        (e_lo + span[0], e_lo + span[1]), int(tun), total_sweeps)


def main(argv=None):
    """Iterate one system to a flat histogram, for one or several walker
    seeds; one JSON line per run and one summary line."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description="iterate one system to a flat histogram")
    ap.add_argument("--system", required=True, help="d:L:N:walkers")
    ap.add_argument("--window", default="0:0", help="simulation window lo:hi (0:0 = [-dN, 0])")
    ap.add_argument("--target", default="", help="flatness target window lo:hi (default: visited range)")
    ap.add_argument("--tempering-target", type=float, default=0.0,
                    help="take the flatness target window from a parallel-tempering run at this "
                         "temperature (Sec. 3): from the energy below which the coldest replicas "
                         "spent 1%% of their time to the highest energy of the replica at T")
    ap.add_argument("--sweeps", type=int, default=1000)
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seeds", type=int, default=1, help="runs with consecutive walker seed blocks")
    ap.add_argument("--scheme", choices=["recursive", "simple"], default="recursive")
    ap.add_argument("--extrapolate", action="store_true",
                    help="or MUCAL_SCHEME_EXTRAPOLATE into the scheme (edge continuation)")
    ap.add_argument("--sweeps-growth", type=int, default=1)
    ap.add_argument("--staged", action="store_true",
                    help="two stages (iterate_staged): range with --range-sweeps, then --sweeps "
                         "measured after --discard discarded sweeps per iteration")
    ap.add_argument("--range-sweeps", type=int, default=1000)
    ap.add_argument("--discard", type=int, default=1000)
    ap.add_argument("--progress", type=int, default=0,
                    help="with --staged: print a JSON line every this many stage-2 iterations")
    args = ap.parse_args(argv)
    d, L, N, W = (int(x) for x in args.system.split(":"))
    lo, hi = (int(x) for x in args.window.split(":"))
    target = [tuple(int(x) for x in args.target.split(":"))] if args.target else None
    temper = None
    if args.tempering_target > 0:
        from . import tempering
        _, _, info = tempering.energy_range(d, L, N, args.tempering_target)
        target = [(info["cold_q01"], info["target_max"])]
        temper = {"T": args.tempering_target, "cold_q01": info["cold_q01"],
                  "target_max": info["target_max"], "cold_min": info["cold_min"]}
    scheme = m.MUCAL_SCHEME_RECURSIVE if args.scheme == "recursive" else m.MUCAL_SCHEME_SIMPLE
    if args.extrapolate:
        scheme |= m.MUCAL_SCHEME_EXTRAPOLATE
    e_lo = -d * N if (lo == 0 and hi == 0) else lo
    rows = []
    for k in range(args.seeds):
        desc = (d, L, N, W, lo, hi, args.seed + k * W)
        if args.staged:
            def report(p, k=k):
                if p["stage2_iteration"] % args.progress == 0:
                    print(json.dumps(dict(p, run=k, flatness=round(p["flatness"], 4))), flush=True)

            r = iterate_staged(desc, range_sweeps=args.range_sweeps, sweeps=args.sweeps,
                               discard=args.discard, max_iter=args.max_iter,
                               target=target[0] if target else None, scheme=scheme,
                               progress=report if args.progress > 0 else None)
            row = {"system": {"d": d, "L": L, "N": N, "walkers": W, "seed_base": desc[-1]},
                   "target": target[0] if target else "sampled range", "tempering": temper,
                   "scheme": args.scheme + (" + edge continuation" if args.extrapolate else ""),
                   "stages": {"range_sweeps": args.range_sweeps, "sweeps": args.sweeps,
                              "discard": args.discard},
                   "iterations": r.iterations, "range_iterations": r.range_iterations,
                   "converged": r.converged, "wall_s": round(r.wall_s, 3),
                   "sampled_range": r.span, "tunnel_events_stage2": r.tunnel_events,
                   "total_sweeps": r.sweeps, "final_flatness": r.flatness[-1],
                   "flatness_every_5": [round(x, 4) for x in r.flatness[::5]]}
            rows.append(row)
            print(json.dumps(row), flush=True)
            continue
        r = iterate_to_flat([desc], args.sweeps, args.max_iter,
                            targets=target, scheme=scheme, sweeps_growth=args.sweeps_growth)[0]
        vis = np.nonzero(r.H > 0)[0]
        row = {"system": {"d": d, "L": L, "N": N, "walkers": W,
                          "window": [e_lo, e_lo + len(r.H) - 1], "seed_base": args.seed + k * W},
               "target": target[0] if target else "visited range", "tempering": temper,
               "sweeps_per_iteration": args.sweeps, "sweeps_last": r.extra["sweeps"][-1],
               "scheme": args.scheme + (" + edge continuation" if args.extrapolate else ""),
               "iterations": r.iterations, "converged": r.converged,
               "wall_s": round(r.wall_s, 3), "attempts": r.attempts,
               "final_flatness": r.flatness[-1] if r.flatness else None,
               "lowest_energy_visited": int(e_lo + vis.min()) if len(vis) else None,
               "flatness_every_10": [round(x, 4) for x in r.flatness[::10]]}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps({"summary": True, "runs": len(rows),
                      "converged": sum(r["converged"] for r in rows),
                      "mean_iterations": float(np.mean([r["iterations"] for r in rows])),
                      "mean_wall_s": float(np.mean([r["wall_s"] for r in rows]))}), flush=True)


if __name__ == "__main__":
    main()
