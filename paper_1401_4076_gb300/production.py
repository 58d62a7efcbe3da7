"""Production run and reweighting to a range of temperatures (Sec. 3).

Once the weights are flat, a production phase with the weights frozen
samples the whole energy range; its histogram, reweighted (Eq. 1), gives the
canonical energy, specific heat and their Ising-equivalent values (Eq. 5) at
every temperature of a grid, and the largest droplet when droplets are
measured.  The iteration runs in the library (walker kernels, histogram sum,
float64 weight update), the droplets are labelled on the device and the
reweighting runs in the library's host code.

    python -m paper_1401_4076_gb300.production --system 2:32:100:1024 \
        --T 0.3:1.5:25 --sweeps 200 --prod 20
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import mucal as m


def run(desc, temperatures, sweeps: int = 200, max_iter: int = 500, goal: float = 0.5,
        prod_rounds: int = 20, prod_sweeps: int = 0, thermal_rounds: int = 2,
        droplets: bool = True, target=None, cuda_stream=None):
    """Iterate desc = (d, L, N, walkers, e_lo, e_hi, seed) to a flat histogram,
    run the production phase and reweight to every T; returns a dict."""
    d, L, N, W, lo, hi, seed = desc
    V = L ** d
    prod_sweeps = prod_sweeps or sweeps
    t0 = time.perf_counter()
    with m.Mucal([desc], cuda_stream=cuda_stream) as mc:
        if target:
            mc.set_target_window(0, *target)
        f = -1.0
        it = 0
        for it in range(max_iter):
            mc.run_iteration(sweeps, it)
            _, f = mc.update_weights(0, m.MUCAL_SCHEME_RECURSIVE)
            if f >= goal:
                break
        iterations = it + 1
        lnW = mc.weights(0)
        info = mc.info[0]
        e_lo = info["e_lo"]
        H = np.zeros(info["n_bins"], dtype=np.int64)
        for r in range(thermal_rounds + prod_rounds):
            mc.run_iteration(prod_sweeps, max_iter + 1 + r)
            if r == thermal_rounds and droplets:
                mc.reset_droplet_stats()
            if r >= thermal_rounds:
                H += mc.histogram(0)
                if droplets:
                    mc.measure_droplets()
        obs = None
        if droplets:
            cnt, s1, _ = mc.droplet_stats(0)
            with np.errstate(invalid="ignore", divide="ignore"):
                obs = np.where(cnt > 0, s1 / np.maximum(cnt, 1), np.nan)[None, :]
    T = np.asarray(temperatures, dtype=np.float64)
    out = m.mucal_reweight(H, lnW, e_lo, 1.0 / T, obs)
    mE, mE2 = out[0], out[1]
    c = m.mucal_ising_constant(d, V, N)
    rows = []
    for i, t in enumerate(T):
        cv = (mE2[i] - mE[i] ** 2) / (t * t * V)
        row = {"T": float(t), "mean_E": float(mE[i]), "specific_heat_per_site": float(cv),
               "T_ising": 4.0 * float(t), "mean_E_ising": 4.0 * (float(mE[i]) - c)}
        if droplets:
            row["mean_V_D"] = float(out[2][i, 0])
        rows.append(row)
    return {"system": {"d": d, "L": L, "N": N, "walkers": W, "window": [e_lo, e_lo + len(H) - 1]},
            "iterations": iterations, "flatness": f, "converged": f >= goal,
            "production_attempts": int(H.sum()), "wall_s": round(time.perf_counter() - t0, 3),
            "curve": rows}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--system", required=True, help="d:L:N:walkers")
    ap.add_argument("--window", default="",
                    help="e_lo:e_hi (0:0 = [-dN, 0]); default: from a tempering run at the "
                         "lowest temperature of the grid")
    ap.add_argument("--T", default="0.3:1.5:25", help="T_min:T_max:points")
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--max-iter", type=int, default=500)
    ap.add_argument("--prod", type=int, default=20, help="production iterations")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    d, L, N, W = (int(x) for x in args.system.split(":"))
    t0, t1, n = args.T.split(":")
    temps = np.linspace(float(t0), float(t1), int(n))
    target = None
    if args.window:
        lo, hi = (int(x) for x in args.window.split(":"))
    else:
        from . import tempering
        lo, hi, info = tempering.energy_range(d, L, N, float(temps.min()), seed=args.seed + 7)
        target = (min(info["target_min"], info["cold_q01"]), info["hot_max"])
    res = run((d, L, N, W, lo, hi, args.seed), temps, sweeps=args.sweeps, max_iter=args.max_iter,
              prod_rounds=args.prod, target=target)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
