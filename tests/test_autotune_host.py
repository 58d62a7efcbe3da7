"""Host logic of the launch-shape autotuner (no GPU): the candidate list it
times.  Every shape the library supports appears, the threshold modes and
the round modes are added only where the kernels have them, and no
candidate is listed twice."""
from paper_1401_4076_gb300 import autotune
from paper_1401_4076_gb300 import mucal as m


def _key(c):
    return tuple(sorted(c.items()))


def test_candidates_cover_every_kernel_and_lane_count():
    cands = autotune.candidates()
    kinds = {(c["kernel"], c["lanes_per_walker"]) for c in cands}
    assert (m.MUCAL_KERNEL_THREAD, 1) in kinds
    for g in (4, 8, 16, 32):
        assert (m.MUCAL_KERNEL_GROUP, g) in kinds
        assert (m.MUCAL_KERNEL_FIELD, g) in kinds
    for c in cands:
        threads = c["lanes_per_walker"] * c["walkers_per_block"]
        assert 1 <= threads <= 1024
        if c["kernel"] != m.MUCAL_KERNEL_THREAD:
            assert threads % 32 == 0          # whole warps per block
        if c["kernel"] == m.MUCAL_KERNEL_FIELD:
            assert c["bits_in_smem"] == 1     # the field lives in shared memory
    assert len({_key(c) for c in cands}) == len(cands)


def test_threshold_and_round_modes_only_where_they_apply():
    base = autotune.candidates()
    out = autotune.with_threshold_modes(base)
    assert len({_key(c) for c in out}) == len(out)
    for c in base:
        assert c in out
    for c in out:
        if c["kernel"] == m.MUCAL_KERNEL_THREAD:
            assert "thr_window" not in c and "multi_commit" not in c
        if c.get("multi_commit"):
            # multi-commit rounds read the rows directly: no row windows, 4+ lanes
            assert c["thr_window"] == 0 and c["lanes_per_walker"] >= 4
    group_field = [c for c in base if c["kernel"] != m.MUCAL_KERNEL_THREAD]
    mc = [c for c in out if c.get("multi_commit")]
    assert len(mc) == sum(1 for c in group_field if c["lanes_per_walker"] >= 4)
    # every group and field shape also with thresholds from global memory
    assert len([c for c in out if c.get("thr_window") == 0 and not c.get("multi_commit")]) == \
        len(group_field)
