"""The weight iteration with its walkers split over processes, on CPU (gloo).

Sec. 2 sums the processes' histograms after every iteration (Eq. 2) and
gives every process the new weights.  Split over ranks, every rank runs its
share of the walkers, the histograms are summed with one int64 all-reduce,
and every rank runs the same double-precision update (the library's
mucal_weight_update, the code its contexts run), so no weights need to be
sent.  Here two ranks each advance half of the walkers of a small system with
the oracle chain (no GPU on this machine), and the summed histogram and the
resulting weights must equal a single process running all walkers with the
same seeds, bit for bit, in every iteration.  The benchmark's helper that
performs the all-reduce for a context is checked against a plain sum too.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

SYSTEM = (2, 8, 12, 16, 0, 0, 100)      # d, L, N, walkers, window (full), seed base
SWEEPS = 40
ITERATIONS = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_iterations(walker_ids, reduce_fn):
    """Advance the given walkers for ITERATIONS iterations; after each, sum
    the histogram with reduce_fn and update the weights in the library.
    Returns the per-iteration (H, lnW)."""
    from oracle import chain
    from paper_1401_4076_gb300 import mucal as m
    d, L, N, W, lo, hi, seed = SYSTEM
    e_lo, e_hi = -d * N, 0
    first = walker_ids[0]
    n = len(walker_ids)
    assert list(walker_ids) == list(range(first, first + n))
    S, occ, E = chain.init_walkers(d, L, N, n, seed + first)
    st = m.WeightState(e_hi - e_lo + 1)
    out = []
    for it in range(ITERATIONS):
        T = chain.thresholds(d, e_lo, e_hi, st.lnW)
        hist, _ = chain.run_walkers(d, L, N, seed + first, it, SWEEPS * N, e_lo, e_hi, T, S, occ, E)
        H = reduce_fn(hist.sum(axis=0))
        m.mucal_weight_update(st, H, m.MUCAL_SCHEME_RECURSIVE)
        out.append((H.copy(), st.lnW.copy()))
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        W = SYSTEM[3]
        share = W // world
        mine = range(rank * share, (rank + 1) * share)

        def allreduce(h):
            t = torch.from_numpy(np.ascontiguousarray(h, dtype=np.int64))
            dist.all_reduce(t)
            return t.numpy().copy()
        res = _run_iterations(mine, allreduce)

        # the benchmark's all-reduce helper on a stand-in context
        import bench

        class FakeContext:
            def __init__(self):
                self.H = [np.arange(7, dtype=np.int64) * (rank + 1),
                          np.full(3, 10 ** 12 + rank, dtype=np.int64)]
                self.given = {}

            def histogram(self, s):
                return self.H[s]

            def set_histogram(self, s, H):
                self.given[s] = np.array(H)
        fc = FakeContext()
        bench.allreduce_histograms(fc, 2, world, "cpu")
        q.put((rank, res, fc.given))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from oracle.build import build_oracle
    from paper_1401_4076_gb300 import _build_ext
    _build_ext.build_library()
    build_oracle()


def test_two_ranks_equal_one_process_bit_for_bit():
    W = SYSTEM[3]
    single = _run_iterations(range(W), lambda h: h)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, res, given = q.get(timeout=300)
        got[rank] = (res, given)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        res, given = got[rank]
        assert len(res) == ITERATIONS
        for (H, lnW), (H1, lnW1) in zip(res, single):
            np.testing.assert_array_equal(H, H1)
            assert np.array_equal(lnW, lnW1)         # identical bits, not just close
        np.testing.assert_array_equal(given[0], np.arange(7) * 3)
        np.testing.assert_array_equal(given[1], np.full(3, 2 * 10 ** 12 + 1))
    # every attempt of every walker is in the summed histogram
    assert single[0][0].sum() == W * SWEEPS * SYSTEM[2]
