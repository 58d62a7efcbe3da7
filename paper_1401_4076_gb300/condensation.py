"""Lattice-gas condensation: the largest droplet against Delta (Sec. 3, Fig. 4).

For a fixed particle number N the density is varied through the lattice size
L.  Each system's energy window comes from a short parallel-tempering run
around the Table 1 temperature (``tempering.energy_range``) unless given;
every system runs the multicanonical iteration of Sec. 2 over its window
until its histogram is flat from the low end of the coldest tempering
replicas to the top of the energies the replica at that temperature visited,
then a production phase with the
weights frozen: after every production iteration the device labels the
clusters of every walker (the largest droplet V_D) and accumulates V_D per
energy.  The histograms and the microcanonical means <V_D>(E) are reweighted
to the temperature of Table 1, and lambda = <V_D> / V_L is set against
Delta of Eq. 10 and the infinite-volume prediction lambda(Delta) (Eq. 9).

All systems of one run share one context and one launch per iteration.
Simulation, labelling, reweighting and the Delta/lambda formulas run in
libmucal; this module only loops and collects.

    python -m paper_1401_4076_gb300.condensation --d 2 --N 100 \
        --deltas 0.4,0.7,1.0,1.5,3 --walkers 1024
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import mucal as m
from . import tempering

# Table 1 (Sec. 3): lattice-gas parameters converted from the Ising model.
TABLE1 = {
    2: {"T": 0.375, "rho0": 0.00675, "kappa_hat": 0.02708, "tau_W": 1.06125},
    3: {"T": 0.500, "rho0": 0.002739, "kappa_hat": 0.00608, "tau_W": 2.861},
}


def delta_of(d: int, L: int, N: int):
    t = TABLE1[d]
    return m.mucal_droplet_delta(d, L ** d, N, t["rho0"], t["kappa_hat"], t["tau_W"])


def sizes_for_deltas(d: int, N: int, deltas, L_max: int = 512):
    """For each wanted Delta the lattice size whose Delta (at this N) is
    closest; duplicates removed, ordered by L."""
    table = []
    for L in range(3, L_max + 1):
        if L ** d <= N:
            continue
        D, vl = delta_of(d, L, N)
        if vl <= 0:
            break
        table.append((L, D))
    out = set()
    for want in deltas:
        out.add(min(table, key=lambda x: abs(x[1] - want))[0])
    return sorted(out)


def run(d: int, N: int, Ls, walkers: int = 1024, sweeps: int = 500, max_iter: int = 1000,
        goal: float = 0.5, prod_rounds: int = 40, prod_sweeps: int = 500, thermal_rounds: int = 5,
        seed: int = 0, windows=None, T=None, keep_rounds=False, cuda_stream=None, log=None):
    """Iterate every system to flatness, then measure; returns one record per L.
    windows: one (e_lo, e_hi) per L, or None to take them from tempering runs.
    T: the temperature to reweight to (default: Table 1's for d; Delta and
    lambda always use Table 1's constants).  keep_rounds: also return every
    production round's histogram and droplet sums (for error estimates)."""
    t = dict(TABLE1[d])
    if T is not None:
        t["T"] = float(T)
    beta = 1.0 / t["T"]
    t0 = time.perf_counter()
    ranges = []
    if windows is None:
        windows = []
        for i, L in enumerate(Ls):
            lo, hi, info = tempering.energy_range(d, L, N, t["T"], seed=seed + 10 ** 6 + 1000 * i,
                                                  cuda_stream=cuda_stream)
            windows.append((lo, hi))
            ranges.append(info)
    t_range = time.perf_counter() - t0
    systems = [(d, L, N, walkers, windows[i][0], windows[i][1], seed + i * walkers)
               for i, L in enumerate(Ls)]
    n = len(systems)
    with m.Mucal(systems, cuda_stream=cuda_stream) as mc:
        # flatness is judged from the energy below which the coldest tempering
        # replicas spent 1 % of their time up to the top of the range the
        # replica at T visited, so a system is not declared converged before
        # its walkers sample the condensed states that matter at T
        for i, info in enumerate(ranges):
            mc.set_target_window(i, min(info["target_min"], info["cold_q01"]), info["target_max"])
        done = [False] * n
        iters = [max_iter] * n
        flat = [-1.0] * n
        it = 0
        for it in range(max_iter):
            mc.run_iteration(sweeps, it)
            for i in range(n):
                if done[i]:
                    continue
                _, f = mc.update_weights(i, m.MUCAL_SCHEME_RECURSIVE)
                flat[i] = f
                if f >= goal:
                    done[i] = True
                    iters[i] = it + 1
            if all(done):
                break
        t_iter = time.perf_counter() - t0
        # production with frozen weights
        lnW = [mc.weights(i) for i in range(n)]
        H = [np.zeros(len(w), dtype=np.int64) for w in lnW]
        rounds = [[] for _ in range(n)]
        prev = [None] * n
        base = max_iter + 1
        for r in range(thermal_rounds + prod_rounds):
            mc.run_iteration(prod_sweeps, base + r)
            if r == thermal_rounds:
                mc.reset_droplet_stats()
            if r >= thermal_rounds:
                for i in range(n):
                    H[i] += mc.histogram(i)
            mc.measure_droplets()
            if keep_rounds and r >= thermal_rounds:
                for i in range(n):
                    st = np.stack(mc.droplet_stats(i))
                    d_st = st if prev[i] is None else st - prev[i]
                    prev[i] = st
                    rounds[i].append((mc.histogram(i), d_st))
        records = []
        stats = []
        for i, L in enumerate(Ls):
            V = L ** d
            cnt, s1, s2 = mc.droplet_stats(i)
            stats.append((cnt, s1, s2))
            with np.errstate(invalid="ignore", divide="ignore"):
                mean_vd = np.where(cnt > 0, s1 / np.maximum(cnt, 1), np.nan)
                mean_vd2 = np.where(cnt > 0, s2 / np.maximum(cnt, 1), np.nan)
            e_lo = windows[i][0] if windows[i] != (0, 0) else -d * N
            mE, mE2, obs = m.mucal_reweight(H[i], lnW[i], e_lo, [beta], np.stack([mean_vd, mean_vd2]))
            D, vl = delta_of(d, L, N)
            vd = float(obs[0, 0])
            rec = {"d": d, "L": L, "N": N, "V": V, "rho": N / V, "T": t["T"],
                   "Delta": D, "V_L": vl, "mean_V_D": vd,
                   "std_V_D": float(np.sqrt(max(obs[0, 1] - vd * vd, 0.0))),
                   "lambda": vd / vl if vl > 0 else None,
                   "lambda_theory": m.mucal_droplet_lambda(d, D),
                   "mean_E": float(mE[0]),
                   # the same state in Ising variables (Eq. 5): T_I = 4T, M = 2N - V
                   "T_ising": 4.0 * t["T"], "M_ising": 2 * N - V,
                   "mean_E_ising": 4.0 * (float(mE[0]) - m.mucal_ising_constant(d, V, N)),
                   "specific_heat_per_site": float(beta ** 2 * (mE2[0] - mE[0] ** 2) / V),
                   "window": [e_lo, e_lo + len(lnW[i]) - 1],
                   "iterations": iters[i], "converged": done[i], "flatness": flat[i],
                   "measurements": int(cnt.sum())}
            if ranges:
                rec["tempering"] = {"cold_min": ranges[i]["cold_min"],
                                    "target_range": [ranges[i]["target_min"], ranges[i]["target_max"]],
                                    "accepted_exchanges": ranges[i]["accepted_exchanges"]}
            records.append(rec)
            if log:
                log(rec)
    wall = time.perf_counter() - t0
    for r in records:
        r["wall_s"] = round(wall, 3)
        r["iteration_wall_s"] = round(t_iter - t_range, 3)
        r["tempering_wall_s"] = round(t_range, 3)
    return records, {"H": H, "lnW": lnW, "droplet_stats": stats, "windows": windows,
                     "rounds": rounds if keep_rounds else None}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="largest droplet against Delta at fixed N")
    ap.add_argument("--d", type=int, default=2)
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--L", default="", help="comma list of lattice sizes (overrides --deltas)")
    ap.add_argument("--deltas", default="0.3,0.6,0.8,0.9,1.0,1.2,1.6,2.5,4")
    ap.add_argument("--walkers", type=int, default=1024)
    ap.add_argument("--sweeps", type=int, default=500,
                    help="sweeps per walker and iteration; near the ground state the walkers "
                         "need hundreds to relax between weight updates")
    ap.add_argument("--max-iter", type=int, default=1000)
    ap.add_argument("--prod-rounds", type=int, default=40)
    ap.add_argument("--prod-sweeps", type=int, default=500)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    if args.L:
        Ls = [int(x) for x in args.L.split(",")]
    else:
        Ls = sizes_for_deltas(args.d, args.N, [float(x) for x in args.deltas.split(",")])
    run(args.d, args.N, Ls, args.walkers, args.sweeps, args.max_iter,
        prod_rounds=args.prod_rounds, prod_sweeps=args.prod_sweeps, seed=args.seed,
        log=lambda r: print(json.dumps(r), flush=True))


if __name__ == "__main__":
    main()
