"""Host logic of the benchmark's multi-process path, on CPU with gloo (world size 2).

Each rank runs an independent copy of the workload (weak scaling): the seed
ranges of the ranks must not overlap, the timing reduction must return the
maximum over ranks, and the CPU reference arm runs on rank 0 only.
"""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_1401_4076_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = workloads.batched_uneven(total_walkers=512)
        mine = bench.shard_systems(wl.systems, rank)
        seeds = set()
        for (d, L, N, W, lo, hi, seed) in mine:
            seeds |= set(range(seed, seed + W))
        t = bench._max_over_ranks(float(rank + 1) * 1.5, world, "cpu")
        w, r, _ = bench._dist_setup()

        class A:
            steps, warmup, gpus = 1, 1, world
        rc = bench.run_reference(A, wl, world, rank) if rank == 1 else 0
        q.put((rank, sorted(seeds), t, w, r, rc))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, seeds, t, w, r, rc = q.get(timeout=120)
        out[rank] = (seeds, t, w, r, rc)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s0, s1 = set(out[0][0]), set(out[1][0])
    assert s0 and s1 and not (s0 & s1)
    assert out[0][1] == out[1][1] == 3.0
    assert out[0][2] == out[1][2] == 2
    assert (out[0][3], out[1][3]) == (0, 1)
    assert out[1][4] == 0          # rank 1 returns without running the reference arm
