"""Host-side rules of bench.py that need no GPU."""
from __future__ import annotations

import bench


def test_traffic_only_for_the_captured_workload_and_tuning():
    t = {"front_words": 2048, "front_kernel": 0}
    assert bench.captured_traffic("projections64", t, "front") == round(
        bench.TRAFFIC_MB[("projections64", 2048, 0)]["front"] * 1e6)
    # another tile size or counting kernel ran other launches: no figure
    assert bench.captured_traffic("projections64", dict(t, front_words=4096), "front") is None
    assert bench.captured_traffic("projections64", dict(t, front_kernel=1), "front") is None
    # a workload without a capture, a stage without a figure
    assert bench.captured_traffic("cube1024", t, "threshold") is None
    assert bench.captured_traffic("projections64", t, "finalize") is None


def test_captured_traffic_is_at_most_a_few_times_the_input():
    # the stages of one step move at most a few times the step's input bytes
    inputs = {"projections64": 241.85, "cube512": 536.87}
    for (wl, _, _), st in bench.TRAFFIC_MB.items():
        assert 0 < sum(st.values()) < 3 * inputs[wl]
