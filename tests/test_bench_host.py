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
    # Philox4x32-10 100, index maps 2, list reads 2, neighbour sites 10d,
    # bit tests 12d, dE and compare 6, histogram 2
    assert bench.alg_ops_per_attempt(2) == 156
    assert bench.alg_ops_per_attempt(3) == 178
