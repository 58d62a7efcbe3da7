"""Host logic of bench.py that needs no GPU: the stored DRAM-traffic record is
reported only for the launch shape and kernel source it was taken with, the
walker-count override only applies to one-system workloads, and the
algorithmic work per attempt is the count the roofline is quoted with."""
import hashlib
import os

import pytest

import bench


def test_traffic_record_matches_only_its_launch_shape_and_source():
    name = "2d-L64-N410-w4096"
    rec = bench.TRAFFIC_MEASURED[name]
    with open(os.path.join(bench.ROOT, "paper_1401_4076_gb300", "csrc", "walker_chain.cuh"), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    launch = dict(rec["launch"], bits_in_smem=1, persistent=0)
    got = bench._measured_traffic(name, True, launch)
    # the record belongs to the current kernel source (else it must read as stale)
    assert got == (rec["bytes"] if sha == rec["kernel_sha"] else None)
    # persistent launches of the same shape run the same blocks
    assert bench._measured_traffic(name, True, dict(launch, persistent=1)) == got
    # another shape, another sweep count or another workload: no figure
    assert bench._measured_traffic(name, True, dict(launch, walkers_per_block=16)) is None
    assert bench._measured_traffic(name, True, dict(launch, kernel=1)) is None
    assert bench._measured_traffic(name, False, launch) is None
    assert bench._measured_traffic("2d-L16-N32-w64", True, launch) is None


def test_walker_override_needs_a_one_system_workload():
    with pytest.raises(SystemExit):
        bench.main(["--workload", "batched", "--walkers", "64"])
    with pytest.raises(SystemExit):
        bench.main(["--walkers", "-3"])


def test_algorithmic_ops_per_attempt():
    # the scope table's count: Philox4x32-10 70 (of 60-80), index maps 2,
    # list reads 2, occupancy bit tests 2 x 2d, threshold 1, histogram 1
    assert bench.alg_ops_per_attempt(2) == 84
    assert bench.alg_ops_per_attempt(3) == 88


def test_headline_is_the_largest_workload():
    """The default workload is the one with the most attempted moves per
    iteration that fits one GPU (the 27-system batch)."""
    sizes = {k: w.attempts_per_iteration() for k, w in bench.WORKLOADS.items()}
    assert max(sizes, key=sizes.get) == "batched"
    import inspect
    src = inspect.getsource(bench.main)
    assert 'default="batched"' in src


def test_instruction_record_follows_shape_and_source():
    rec = {"x": {"launch": {"kernel": 1, "lanes_per_walker": 4}, "kernel_sha": bench._kernel_sha(),
                 "warp_inst_per_attempt": 100.0, "thread_inst_per_attempt": 900.0}}
    assert bench._record_for(rec, "x", True, {"kernel": 1, "lanes_per_walker": 4}) is rec["x"]
    assert bench._record_for(rec, "x", True, {"kernel": 1, "lanes_per_walker": 8}) is None
    assert bench._record_for(rec, "x", False, {"kernel": 1, "lanes_per_walker": 4}) is None
    rec["x"]["kernel_sha"] = "0" * 16
    assert bench._record_for(rec, "x", True, {"kernel": 1, "lanes_per_walker": 4}) is None


def test_records_per_round_mode():
    """A workload may hold one record per launch variant (the 3D workload:
    multi-commit and one-commit rounds); the launch picks its own."""
    name = "3d-L32-N3277-w8192"
    recs = bench.TRAFFIC_MEASURED[name]
    assert isinstance(recs, list) and len(recs) == 2
    base = dict(kernel=1, lanes_per_walker=4, walkers_per_block=56, bits_in_smem=1,
                persistent=1, thr_window=0)
    current = recs[0]["kernel_sha"] == bench._kernel_sha()
    for mc, rec in ((1, recs[0]), (0, recs[1])):
        assert rec["launch"]["multi_commit"] == mc
        got = bench._measured_traffic(name, True, dict(base, multi_commit=mc))
        assert got == (rec["bytes"] if current else None)
    assert bench._measured_traffic(name, True, dict(base, multi_commit=1, thr_window=1)) is None


def test_reference_arm_line(capsys):
    """`--impl reference` on rank 0: one JSON line timing the oracle on a
    bounded sample of the workload, with the keys the line must carry."""
    import json
    from paper_1401_4076_gb300 import workloads

    class A:
        steps, warmup, gpus, sweeps = 1, 1, 1, 0

    wl = workloads.batched_uneven(total_walkers=256)
    assert bench.run_reference(A, wl, 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "attempts/s" and line["higher_is_better"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "walkers" in cb["sample"] and "sweeps" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "attempts/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == wl.name
