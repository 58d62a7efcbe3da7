"""Multicanonical reweighting against direct canonical simulation (Sec. 4,
Fig. 2).

The paper checks its parallel multicanonical lattice-gas results against
micromagnetic (fixed-magnetisation Metropolis) simulations of the Ising model
at the same temperature, on L = 30 in three dimensions with the particle
number varied.  By Eq. 5 the fixed-magnetisation Ising model is the fixed-N
lattice gas with T_Ising = 4 T, so the direct simulation here is canonical
Metropolis of the lattice gas itself (weights lnW(E) = -E/T, the same walker
kernels), many independent walkers, averages over iterations after a
thermalisation, error bars from batch means.  The multicanonical side is the
pipeline of ``condensation.run`` (tempering window, iteration to a flat
histogram, production, reweighting to T).

    python -m paper_1401_4076_gb300.compare --d 3 --L 30 --T 0.6995 \
        --N 200,400,600,800,1000,1200
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import condensation
from . import mucal as m


def canonical(d: int, L: int, N: int, T: float, walkers: int = 4096, sweeps: int = 20,
              thermal: int = 100, measure: int = 200, batches: int = 10, seed: int = 0,
              cuda_stream=None):
    """<E> and <V_D> of canonical Metropolis at temperature T with their
    batch-mean errors."""
    beta = 1.0 / T
    e_lo = -d * N
    grid = np.arange(e_lo, 1, dtype=np.float64)
    e_means, d_means = [], []
    t0 = time.perf_counter()
    with m.Mucal([(d, L, N, walkers, 0, 0, seed)], cuda_stream=cuda_stream) as mc:
        mc.set_weights(0, -beta * grid)
        for it in range(thermal):
            mc.run_iteration(sweeps, it)
        per = measure // batches
        for b in range(batches):
            H = np.zeros(len(grid), dtype=np.int64)
            vd = 0.0
            for k in range(per):
                mc.run_iteration(sweeps, thermal + b * per + k)
                H += mc.histogram(0)
                mc.measure_droplets()
                vd += float(mc.largest_droplets(0).mean())
            e_means.append(float((H * grid).sum() / H.sum()))
            d_means.append(vd / per)
    err = lambda x: float(np.std(x, ddof=1) / math.sqrt(len(x)))
    return {"mean_E": float(np.mean(e_means)), "err_E": err(e_means),
            "mean_V_D": float(np.mean(d_means)), "err_V_D": err(d_means),
            "attempts": walkers * sweeps * N * (thermal + measure),
            "wall_s": round(time.perf_counter() - t0, 3)}


def muca_jackknife(aux, d: int, N: int, T: float, blocks: int = 10):
    """Jackknife errors of the reweighted <E> and <V_D> over blocks of
    production rounds (each leave-one-block-out set reweighted afresh)."""
    rounds = aux["rounds"][0]
    lnW = aux["lnW"][0]
    e_lo = aux["windows"][0][0] if tuple(aux["windows"][0]) != (0, 0) else -d * N
    beta = 1.0 / T
    size = max(1, len(rounds) // blocks)
    groups = [rounds[k * size:(k + 1) * size] for k in range(len(rounds) // size)]
    H_all = np.sum([h for grp in groups for (h, _) in grp], axis=0)
    D_all = np.sum([st for grp in groups for (_, st) in grp], axis=0)
    est = []
    for grp in groups:
        H = H_all - np.sum([h for (h, _) in grp], axis=0)
        D = D_all - np.sum([st for (_, st) in grp], axis=0)
        with np.errstate(invalid="ignore", divide="ignore"):
            vd = np.where(D[0] > 0, D[1] / np.maximum(D[0], 1), np.nan)
        mE, _, obs = m.mucal_reweight(H, lnW, e_lo, [beta], vd[None, :])
        est.append((float(mE[0]), float(obs[0, 0])))
    est = np.array(est)
    k = len(est)
    err = np.sqrt((k - 1) / k * ((est - est.mean(axis=0)) ** 2).sum(axis=0))
    return float(err[0]), float(err[1])


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--L", type=int, default=30)
    ap.add_argument("--T", type=float, default=0.6995)
    ap.add_argument("--N", default="200,400,600,800,1000,1200")
    ap.add_argument("--walkers", type=int, default=1024)
    ap.add_argument("--canonical-walkers", type=int, default=4096)
    ap.add_argument("--max-iter", type=int, default=1000)
    args = ap.parse_args(argv)
    for i, N in enumerate(int(x) for x in args.N.split(",")):
        recs, aux = condensation.run(args.d, N, [args.L], walkers=args.walkers,
                                     max_iter=args.max_iter, T=args.T, seed=1000 * i,
                                     keep_rounds=True)
        r = recs[0]
        eE, eV = muca_jackknife(aux, args.d, N, args.T)
        c = canonical(args.d, args.L, N, args.T, walkers=args.canonical_walkers, seed=10 ** 7 + i)
        print(json.dumps({"d": args.d, "L": args.L, "N": N, "T": args.T,
                          "muca": {"mean_E": r["mean_E"], "err_E": eE,
                                   "mean_V_D": r["mean_V_D"], "err_V_D": eV,
                                   "iterations": r["iterations"], "converged": r["converged"],
                                   "window": r["window"], "wall_s": r["wall_s"]},
                          "canonical": c,
                          "dE_in_err": (r["mean_E"] - c["mean_E"]) / max(math.hypot(eE, c["err_E"]), 1e-12),
                          "dVD_in_err": (r["mean_V_D"] - c["mean_V_D"]) /
                          max(math.hypot(eV, c["err_V_D"]), 1e-12)}),
              flush=True)


if __name__ == "__main__":
    main()
