"""Host-side rules of bench.py that need no GPU."""
from __future__ import annotations

import bench


def test_traffic_carries_the_launch_shape_of_its_capture(monkeypatch):
    shape = {"front_words": 2048, "front_kernel": 0}
    table = {"projections64": {"front": 128.2, "tuning": shape, "source": "ncu capture X"}}
    monkeypatch.setattr(bench, "TRAFFIC_MB", table)
    t = dict(shape, thr_blocks_per_sm=8)
    assert bench.captured_traffic("projections64", t, "front") == (128200000, "ncu capture X", None)
    # another tile size or counting kernel: the figure, with the capture's shape
    for other in (dict(t, front_words=4096), dict(t, front_kernel=1)):
        assert bench.captured_traffic("projections64", other, "front") == (
            128200000, "ncu capture X", shape)
    # a workload without a capture, a stage without a figure
    assert bench.captured_traffic("cube1024", t, "threshold") == (None, None, None)
    assert bench.captured_traffic("projections64", t, "finalize") == (None, None, None)


def test_captured_traffic_is_at_most_a_few_times_the_input():
    # the stages of one step move at most a few times the step's input bytes
    inputs = {"projections64": 241.85, "cube512": 536.87, "cube1024": 4294.97}
    for wl, st in bench.TRAFFIC_MB.items():
        assert isinstance(st["source"], str) and st["source"]
        assert set(st["tuning"]) <= {"front_words", "front_kernel"}
        vals = [v for k, v in st.items() if k not in ("source", "tuning")]
        assert 0 < sum(vals) < 3 * inputs[wl]


def test_sub_line_keeps_the_measurement_fields():
    m = {"value": 1234.567, "ms_per_step": 0.123456, "in_bytes": 1000, "out_bytes": 100,
         "latency": {"p50_ms": 1}, "clocks": {"sm_mhz": 2070}, "roofline": {"frac": 0.5},
         "tuning": {"front_words": 2048}, "launches_per_step": 12, "nstreams": 8, "graph": True}
    line = bench.sub_line(m, [0, 1], {}, "d", bench.path_text("plain", m))
    assert line["value"] == 1234.57 and line["ms_per_step"] == 0.1235
    assert line["compression_ratio"] == 10.0 and line["items"] == 2
    assert line["path"] == "roix_compress per item on 8 streams, one CUDA graph per step"
    for k in ("latency", "clocks", "roofline", "tuning"):
        assert line[k] == m[k]



def _shaped(shape, dtype):
    import torch
    # a view of one element: shape, element size and an aligned pointer, no storage
    return torch.empty(1, dtype=dtype).expand(*shape)


def test_launch_count_rules_match_the_profiled_launch_lists():
    import torch
    import phantom
    # 64 uint16 projections 512..2048 wide: the flat binarisation, no scans —
    # the nine kernels of one step in the ncu launch list of that workload
    xs = [_shaped((s, s), torch.uint16) for s in phantom.projection_sides(64, 512, 2048, 0)]
    assert bench.group_launches(xs) == 9
    # the 1024^3 float32 volume: the row form, the compaction's tile scan, the
    # pack's chunk scan and records — twelve kernels in its launch list
    assert bench.group_launches([_shaped((1024, 1024, 1024), torch.float32)]) == 12
    # a small volume: no scan launches; 1024-voxel rows take the row form
    assert bench.group_launches([_shaped((16, 64, 1024), torch.float32)]) == 9
    # a larger tile (front_words) halves the tiles, not the chunks
    assert bench.group_launches([_shaped((1024, 1024, 1024), torch.float32)],
                                tuning={"front_words": 16384}) == 12
