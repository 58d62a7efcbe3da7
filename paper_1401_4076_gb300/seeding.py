"""Learned seeding of the multicanonical weights (not part of the paper).

The iteration of Sec. 2 starts from some W^0 and improves it with every
histogram; W = 1/Omega is its fixed point.  This module trains the library's
GPU network on ln Omega estimates that converged runs of the method itself
produced on small lattices, and uses it to propose W^0 = 1/Omega_pred for a
larger lattice.  The proposal only changes where the iteration starts (and, after a seed,
the update uses the memory-free simple scheme of Sec. 2): the walkers and
the flatness judgement are unchanged, and the plain start lnW = 0 with the
recursion remains available as fallback and reference.

Network input: (d, L, rho, E/V), encoded as
    x = (2 (d - 2.5), 16 / L, 10 rho - 0.5, 2 (E/V) / (d rho) + 1);
output: ln Omega(E) / V divided by the ideal-gas entropy density
ln C(V, N) / V, i.e. ln Omega(E) / ln C(V, N), a number in [0, 1].

All simulation and training runs in libmucal on the GPU; this module only
arranges inputs and collects results.
"""
from __future__ import annotations

import time

import numpy as np

from . import mucal as m
from .iterate import (RunResult, iterate_staged, iterate_to_flat, ln_binomial,  # noqa: F401
                      ln_omega_estimate)


def features(d: int, L: int, N: int, E: np.ndarray) -> np.ndarray:
    """Network inputs for energies E of a d-dimensional L^d lattice with N particles."""
    V = L ** d
    rho = N / V
    e = np.asarray(E, dtype=np.float64) / V
    X = np.empty((len(e), 4), dtype=np.float32)
    X[:, 0] = 2.0 * (d - 2.5)
    X[:, 1] = 16.0 / L
    X[:, 2] = 10.0 * rho - 0.5
    X[:, 3] = 2.0 * e / (d * rho) + 1.0
    return X


def training_set(results):
    """(X, t) rows from converged runs: every visited bin of the final
    histogram with its ln Omega estimate, normalised by ln C(V, N)."""
    Xs, ts = [], []
    for r in results:
        d, L, N, W, lo, hi, seed = r.desc
        V = L ** d
        e_lo = -d * N if (lo == 0 and hi == 0) else lo
        lo_est = ln_omega_estimate(r.lnW, r.H, V, N)
        ok = ~np.isnan(lo_est)
        E = e_lo + np.nonzero(ok)[0]
        Xs.append(features(d, L, N, E))
        ts.append((lo_est[ok] / ln_binomial(V, N)).astype(np.float32))
    return np.concatenate(Xs), np.concatenate(ts)


def train(X, t, steps: int = 3000, lr: float = 2e-3, seed: int = 0, cuda_stream=None,
          final_lr_fraction: float = 0.05):
    """Train the GPU network (full-batch Adam in the library) and return it.
    The learning rate decays geometrically in chunks of 500 steps from lr to
    final_lr_fraction * lr, so that training ends in a settled minimum."""
    from .workloads import mlp_initial_params
    net = m.Mlp(mlp_initial_params(seed), cuda_stream=cuda_stream)
    loss = None
    done = 0
    chunks = max(1, (steps + 499) // 500)
    for c in range(chunks):
        k = min(500, steps - done)
        rate = lr * final_lr_fraction ** (c / max(1, chunks - 1))
        loss = net.train(X, t, steps=k, lr=rate)
        done += k
    return net, loss


def seed_weights(net, d: int, L: int, N: int, e_lo: int, e_hi: int) -> np.ndarray:
    """lnW^0(E) = -ln Omega_pred(E) over the window, shifted to max 0."""
    E = np.arange(e_lo, e_hi + 1)
    y = net.forward(features(d, L, N, E)).astype(np.float64)
    lnW = -y * ln_binomial(L ** d, N)
    return lnW - lnW.max()


def window_fraction(d: int, N: int, frac: float):
    """Energy window [-frac * d * N, 0]: the upper part of the full range
    [-dN, 0], from the gas side down to frac of the maximal bond count."""
    return (-int(frac * d * N), 0)


def small_training_systems(frac: float = 0.5, walkers: int = 512, seed_base: int = 0,
                           L2=(12, 16, 20, 24, 28, 32, 40), L3=(6, 8, 10, 12, 14),
                           rhos=(0.05, 0.07, 0.09, 0.1, 0.11, 0.13)):
    """Descriptors of the small systems whose converged weights train the network."""
    out = []
    seed = seed_base
    for d, Ls in ((2, L2), (3, L3)):
        for L in Ls:
            for rho in rhos:
                N = int(round(rho * L ** d))
                lo, hi = window_fraction(d, N, frac)
                out.append((d, L, N, walkers, lo, hi, seed))
                seed += walkers
    return out


def compare_plain_and_seeded(net, desc, sweeps: int, max_iter: int, relax_iters: int = 30,
                             relax_tol: float = 0.002, seeded_scheme=m.MUCAL_SCHEME_SIMPLE,
                             cuda_stream=None, plain_scheme=m.MUCAL_SCHEME_RECURSIVE):
    """Iterations and wall time to flatness from lnW = 0 with plain_scheme
    (the plain method, the reference) and from the network's seed, same
    system, seeds, sweeps and window.

    The seeded run updates with the simple scheme W/H: its first histograms
    come from walkers still relaxing towards the seeded weights, and the
    simple scheme keeps no memory of them, whereas the accumulated-statistics
    recursion would carry their bias for many iterations (measured: the
    recursive scheme after a seed is slower than either plain start)."""
    d, L, N, W, lo, hi, seed = desc
    seedW = seed_weights(net, d, L, N, lo, hi)
    plain = iterate_to_flat([desc], sweeps, max_iter, scheme=plain_scheme, cuda_stream=cuda_stream)[0]
    seeded = iterate_to_flat([desc], sweeps, max_iter, lnW0=[seedW], relax_iters=relax_iters,
                             relax_tol=relax_tol, scheme=seeded_scheme, cuda_stream=cuda_stream)[0]
    return plain, seeded, seedW


def compare_staged(net, desc, **kw):
    """The two-stage iteration (iterate_staged) from lnW = 0 and from the
    network's seed, same system, walker seeds and stage parameters; the seed
    replaces stage 1 by a relaxation with the seeded weights held fixed.
    Both are judged on the same target window: the one given, else the
    range the plain run's stage 1 sampled.  Returns (plain, seeded, seed
    weights)."""
    d, L, N, W, lo, hi, seed = desc
    e_lo, e_hi = (-d * N, 0) if (lo == 0 and hi == 0) else (lo, hi)
    seedW = seed_weights(net, d, L, N, e_lo, e_hi)
    seed_range_stage = kw.pop("seed_range_stage", False)
    plain = iterate_staged(desc, **kw)
    if kw.get("target") is None:
        kw = dict(kw, target=plain.span)
    seeded = iterate_staged(desc, lnW0=seedW, seed_range_stage=seed_range_stage, **kw)
    return plain, seeded, seedW


def ladder(net, rungs, frac: float, walkers: int, sweeps: int, max_iter: int, X, t,
           train_steps: int = 5000, compare: bool = True, log=None, seed_base: int = 10 ** 7):
    """Climb in lattice size: seed each rung from the current network, run the
    iteration to flatness, add the converged ln Omega estimate to the training
    rows and continue training (warm start) before the next rung.  Every rung
    is trained only on smaller lattices.  Returns (network, records)."""
    records = []
    for k, (d, L, rho) in enumerate(rungs):
        N = int(round(rho * L ** d))
        lo, hi = window_fraction(d, N, frac)
        desc = (d, L, N, walkers, lo, hi, seed_base + k * walkers)
        seedW = None
        if compare:
            plain, seeded, seedW = compare_plain_and_seeded(net, desc, sweeps, max_iter)
        else:
            plain = None
            seeded = iterate_to_flat([desc], sweeps, max_iter,
                                     lnW0=[seed_weights(net, d, L, N, lo, hi)],
                                     relax_iters=30, relax_tol=0.002,
                                     scheme=m.MUCAL_SCHEME_SIMPLE)[0]
        rec = {"system": {"d": d, "L": L, "N": N, "walkers": walkers, "window": [lo, hi],
                          "sweeps_per_iteration": sweeps},
               "seeded": {"iterations": seeded.iterations, "converged": seeded.converged,
                          "wall_s": round(seeded.wall_s, 3), "flatness": seeded.flatness[-1],
                          "relax_iterations": int(np.isnan(seeded.flatness).sum())}}
        if plain is not None:
            rec["plain"] = {"iterations": plain.iterations, "converged": plain.converged,
                            "wall_s": round(plain.wall_s, 3), "flatness": plain.flatness[-1]}
            if plain.converged:
                # seed error against the weights the plain run converged to
                diff = seedW - plain.lnW
                rec["seed_error"] = {"range": round(float(np.ptp(diff)), 3),
                                     "slope_rms": round(float(np.sqrt(np.mean(np.diff(diff) ** 2))), 4)}
        records.append(rec)
        if log:
            log(rec)
        if seeded.converged:
            # a longer run at the converged weights for the ln Omega estimate
            fin = iterate_to_flat([desc], sweeps, 1, lnW0=[seeded.lnW], relax_iters=0,
                                  final_sweeps=4 * sweeps, goal=2.0)[0]
            Xk, tk = training_set([RunResult(desc, 0, [], True, 0.0, seeded.lnW, fin.H)])
            X = np.concatenate([X, Xk])
            t = np.concatenate([t, tk])
            params = net.params()
            net.close()
            net = m.Mlp(params)
            done = 0
            while done < train_steps:
                step = min(500, train_steps - done)
                net.train(X, t, steps=step, lr=5e-4)
                done += step
    return net, records


def full_range_trials(trainings: int, seeds: int, train_steps: int, log):
    """The plain start against the learned seed on 2D L=64, N=410, 4096
    walkers over its whole sampled range (two-stage iteration, flatness
    over [-778, 0]), with the network trained `trainings` times on the same
    rows.  On the tensor cores (the default) the training's sums run in a
    fixed order, so every training gives the same network and the repeats
    check that; with the mma.sync path (atomic sums) they differ slightly.
    The plain runs are the same for every training (the chain is
    deterministic) and run once per seed."""
    from .iterate import iterate_staged
    scheme = m.MUCAL_SCHEME_SIMPLE | m.MUCAL_SCHEME_EXTRAPOLATE
    small = small_training_systems(1.0)
    res = iterate_to_flat(small, sweeps=100, max_iter=300, final_sweeps=1000, scheme=scheme)
    X, t = training_set([r for r in res if r.converged])
    d, L, N, W = 2, 64, 410, 4096
    walker_seeds = [7 * 10 ** 6 + k * W for k in range(seeds)]
    for k, s in enumerate(walker_seeds):
        r = iterate_staged((d, L, N, W, 0, 0, s), max_iter=150, target=(-778, 0))
        log({"start": "plain", "seed": k, "iterations": r.iterations,
             "wall_s": round(r.wall_s, 2), "converged": r.converged})
    for rep in range(trainings):
        t0 = time.perf_counter()
        net, loss = train(X, t, steps=train_steps, lr=1e-3)
        tt = time.perf_counter() - t0
        seedW = seed_weights(net, d, L, N, -d * N, 0)
        for k, s in enumerate(walker_seeds):
            r = iterate_staged((d, L, N, W, 0, 0, s), lnW0=seedW, max_iter=150, target=(-778, 0))
            log({"start": "learned", "training": rep, "train_s": round(tt, 2), "loss": loss,
                 "seed": k, "iterations": r.iterations, "wall_s": round(r.wall_s, 2),
                 "converged": r.converged})
        net.close()


def main(argv=None):
    """Train on small systems, then compare plain and seeded convergence on
    larger ones; prints one JSON line per target system."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--frac", type=float, default=0.5)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--targets", default="2:48:0.1:4096:50,2:64:0.1:4096:50,2:96:0.1:4096:50,"
                    "3:16:0.1:4096:50,3:20:0.1:4096:50",
                    help="comma list of d:L:rho:walkers:sweeps")
    ap.add_argument("--max-iter", type=int, default=300)
    ap.add_argument("--relax", type=int, default=30, help="cap on relaxation iterations")
    ap.add_argument("--relax-tol", type=float, default=0.002)
    ap.add_argument("--ladder", default="",
                    help="rungs d:L:rho separated by commas, climbed after training")
    ap.add_argument("--ladder-walkers", type=int, default=4096)
    ap.add_argument("--ladder-sweeps", type=int, default=50)
    ap.add_argument("--full-range-trainings", type=int, default=0,
                    help="train the network this many times on small lattices run over their "
                         "whole ranges, and compare the two-stage iteration from lnW = 0 and "
                         "from each network's seed on 2D L=64, N=410, 4096 walkers (flatness "
                         "over [-778, 0])")
    ap.add_argument("--full-range-seeds", type=int, default=4,
                    help="walker seeds of that comparison")
    ap.add_argument("--train-steps-only", type=int, default=0,
                    help="only run this many training steps of the network on the 8192-row "
                         "test batch (a fixed workload for profiling the training kernels)")
    args = ap.parse_args(argv)
    if args.train_steps_only:
        from .workloads import mlp_initial_params, mlp_test_batch
        X, t = mlp_test_batch(8192, 1)
        with m.Mlp(mlp_initial_params(0)) as net:
            loss = net.train(X, t, steps=args.train_steps_only, lr=1e-3)
        print(json.dumps({"train_steps": args.train_steps_only, "rows": 8192, "loss": loss}))
        return
    if args.full_range_trainings:
        full_range_trials(args.full_range_trainings, args.full_range_seeds, args.train_steps,
                          lambda r: print(json.dumps(r), flush=True))
        return
    t0 = time.perf_counter()
    small = small_training_systems(args.frac)
    res = iterate_to_flat(small, sweeps=100, max_iter=200, final_sweeps=1000)
    X, t = training_set([r for r in res if r.converged])
    t_runs = time.perf_counter() - t0
    t1 = time.perf_counter()
    net, loss = train(X, t, steps=args.train_steps, lr=1e-3)
    print(json.dumps({"training_systems": len(small),
                      "converged": int(sum(r.converged for r in res)), "rows": int(len(t)),
                      "training_runs_s": round(t_runs, 3),
                      "network_training_s": round(time.perf_counter() - t1, 3),
                      "final_loss": loss}))
    if args.ladder:
        rungs = []
        for spec in args.ladder.split(","):
            d, L, rho = spec.split(":")
            rungs.append((int(d), int(L), float(rho)))
        net, _ = ladder(net, rungs, args.frac, args.ladder_walkers, args.ladder_sweeps,
                        args.max_iter, X, t, log=lambda r: print(json.dumps({"rung": r}), flush=True))
        net.close()
        return
    for spec in args.targets.split(","):
        d, L, rho, W, sweeps = spec.split(":")
        d, L, W, sweeps = int(d), int(L), int(W), int(sweeps)
        N = int(round(float(rho) * L ** d))
        lo, hi = window_fraction(d, N, args.frac)
        desc = (d, L, N, W, lo, hi, 10 ** 6)
        plain, seeded, seedW = compare_plain_and_seeded(net, desc, sweeps, args.max_iter, args.relax,
                                                        args.relax_tol)
        print(json.dumps({"system": {"d": d, "L": L, "N": N, "walkers": W, "window": [lo, hi],
                                     "sweeps_per_iteration": sweeps},
                          "plain": {"iterations": plain.iterations, "converged": plain.converged,
                                    "wall_s": round(plain.wall_s, 3),
                                    "flatness": plain.flatness[-1]},
                          "seeded": {"iterations": seeded.iterations,
                                     "converged": seeded.converged,
                                     "wall_s": round(seeded.wall_s, 3),
                                     "flatness": seeded.flatness[-1],
                                     "relax_iterations": int(sum(np.isnan(seeded.flatness)))}}))
    net.close()


if __name__ == "__main__":
    main()
