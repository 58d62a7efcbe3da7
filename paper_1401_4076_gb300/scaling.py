"""Iterations and time to convergence against the number of walkers (Sec. 4,
Fig. 3).

The paper fixes the total work of one iteration (25 600 sweeps of L^d
updates, each of the p processes doing 25600/p of them), declares a run
converged once its processes together have made 30 tunnelling events
(travels between the lowest and the highest energy of the range), and
reports the mean number of iterations and the speed-up S_p = t_1 / t_p over
independent runs.  Here the p processes are p walkers of one system on the
GPU; the tunnelling events are counted inside the walker kernels.  Every
run uses its own context, so its wall time is that of the run alone.

    python -m paper_1401_4076_gb300.scaling --d 2 --N 100 --L 74 \
        --walkers 1,4,16,64,256,1024,4096 --seeds 4
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import mucal as m


def converge(desc, total_sweeps: int, max_iter: int = 500, events: int = 30, launch=None,
             scheme=m.MUCAL_SCHEME_RECURSIVE, cuda_stream=None):
    """One run: iterate the weights until the walkers' tunnelling events
    reach `events`.  Each walker performs total_sweeps / p sweeps of V
    updates per iteration.  Returns a result dict."""
    d, L, N, p, lo, hi, seed = desc
    V = L ** d
    attempts = max(1, int(round(total_sweeps * V / p)))
    sweeps = max(1, int(round(attempts / N)))      # the library counts sweeps of N attempts
    t0 = time.perf_counter()
    with m.Mucal([desc], cuda_stream=cuda_stream) as mc:
        if launch:
            mc.set_launch(**launch)
        mc.set_tunnel_window(0, 0, 0)            # events between the window's ends
        total = 0
        it = 0
        for it in range(max_iter):
            mc.run_iteration(sweeps, it)
            mc.update_weights(0, scheme)
            total = mc.tunnel_counts(0)[0]
            if total >= events:
                break
        wall = time.perf_counter() - t0
    return {"walkers": p, "seed": seed, "iterations": it + 1, "converged": total >= events,
            "events": int(total), "wall_s": wall, "sweeps_per_walker": sweeps * N / V}


def launch_for(p: int):
    """Lanes per walker: many lanes when few walkers leave the GPU idle."""
    if p < 256:
        return dict(kernel=m.MUCAL_KERNEL_GROUP, lanes_per_walker=32, walkers_per_block=4,
                    bits_in_smem=1)
    return None


def study(d: int, L: int, N: int, window, walkers, seeds: int, total_sweeps: int,
          max_iter: int, events: int = 30, log=None):
    lo, hi = window
    rows = []
    for p in walkers:
        runs = [converge((d, L, N, p, lo, hi, 1000003 * s + 17), total_sweeps, max_iter, events,
                         launch_for(p)) for s in range(seeds)]
        row = {"walkers": p, "runs": len(runs),
               "converged": int(sum(r["converged"] for r in runs)),
               "iterations_mean": float(np.mean([r["iterations"] for r in runs])),
               "iterations_std": float(np.std([r["iterations"] for r in runs])),
               "wall_s_mean": float(np.mean([r["wall_s"] for r in runs])),
               "sweeps_per_walker": runs[0]["sweeps_per_walker"]}
        rows.append(row)
        # speed-up relative to the first walker count
        row["speedup_S_p"] = rows[0]["wall_s_mean"] / row["wall_s_mean"]
        row["iteration_ratio"] = rows[0]["iterations_mean"] / row["iterations_mean"]
        if log:
            log(row)
    return rows


def main(argv=None):
    import argparse
    from . import tempering
    from .condensation import TABLE1
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--L", type=int, default=74)
    ap.add_argument("--walkers", default="1,4,16,64,256,1024,4096")
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--total-sweeps", type=int, default=2560,
                    help="sweeps of L^d updates per iteration, shared by the walkers")
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--events", type=int, default=30)
    ap.add_argument("--window", default="", help="lo:hi (default: from tempering at the Table 1 T)")
    args = ap.parse_args(argv)
    if args.window:
        window = tuple(int(x) for x in args.window.split(":"))
    else:
        lo, hi, info = tempering.energy_range(args.d, args.L, args.N, TABLE1[args.d]["T"], seed=7)
        window = (lo, hi)
    print(json.dumps({"system": {"d": args.d, "L": args.L, "N": args.N, "window": list(window)},
                      "total_sweeps_per_iteration": args.total_sweeps, "events": args.events}),
          flush=True)
    study(args.d, args.L, args.N, window, [int(x) for x in args.walkers.split(",")], args.seeds,
          args.total_sweeps, args.max_iter, args.events, log=lambda r: print(json.dumps(r), flush=True))


if __name__ == "__main__":
    main()
