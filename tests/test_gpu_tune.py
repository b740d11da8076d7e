"""Autotuner (roix_tune) and launch-shape settings, through the C ABI.

The tuned values only change launch shapes: every container must stay the
oracle's byte for byte under any setting, the tuner must pick values from its
candidate lists, and a cached entry must be applied again without timing.
"""
from __future__ import annotations

import json
import time

import numpy as np
import pytest
import torch

import oracle
import phantom

pytestmark = pytest.mark.gpu

CFG16 = dict(eb=4, eb_mode="abs", cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
CFG32 = dict(eb=1e-4, eb_mode="rel", threshold=0.1, dilate=1)


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    r = roix.Roix(0)
    yield r
    r.close()


def _check_batch(rx, xs, cfg):
    outs, sizes = rx.compress_batch(xs, **cfg)
    rx.sync()
    for x, o, sz in zip(xs, outs, sizes.cpu().numpy()):
        ref = oracle.compress(x.cpu().numpy(), **cfg)
        got = o[:int(sz)].cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref)


@pytest.mark.parametrize("setting", [
    dict(front_words=256), dict(front_words=16384), dict(thr_blocks_per_sm=1, flat_blocks_per_sm=1),
    dict(thr_blocks_per_sm=32, flat_blocks_per_sm=32), dict(sym_blocks_per_sm=1, pack_blocks_per_sm=1),
    dict(sym_blocks_per_sm=32, pack_blocks_per_sm=32), dict(front_kernel=1),
    dict(front_kernel=1, front_words=256), dict(front_kernel=1, front_words=16384)])
def test_any_setting_keeps_the_bytes(rx, setting):
    default = rx.get_tuning()
    try:
        rx.set_tuning(**setting)
        xs = [phantom.projection(s, i, seed=3, device="cuda") for i, s in enumerate([300, 512, 777])]
        _check_batch(rx, xs, CFG16)
        x = phantom.porous_cylinder(80, radius=30, seed=4, device="cuda")
        _check_batch(rx, [x], CFG32)
    finally:
        rx.set_tuning(**default)


def test_set_tuning_rejects_out_of_range(rx):
    import paper_2602_15917_gb300 as roix
    before = rx.get_tuning()
    for bad in (dict(front_words=100), dict(thr_blocks_per_sm=0), dict(pack_blocks_per_sm=33),
                dict(front_kernel=2)):
        with pytest.raises(roix.RoixError) as ei:
            rx.set_tuning(**bad)
        assert ei.value.status == 1
    assert rx.get_tuning() == before


def test_tune_picks_candidates_caches_and_keeps_bytes(rx, tmp_path):
    import paper_2602_15917_gb300 as roix
    cache = str(tmp_path / "tune.json")
    xs = [phantom.projection(s, i, seed=5, device="cuda") for i, s in enumerate([640, 901, 1024])]
    t = rx.tune(xs, reps=3, cache=cache, **CFG16)
    assert t["front_words"] in (512, 1024, 2048, 4096, 8192)
    assert t["thr_blocks_per_sm"] in (2, 4, 8, 16)
    assert t["flat_blocks_per_sm"] in (2, 3, 4, 8)
    assert t["sym_blocks_per_sm"] in (0, 1, 2, 3)
    assert t["pack_blocks_per_sm"] in (0, 1, 2, 4)
    assert t["front_kernel"] in (0, 1)
    assert rx.get_tuning() == t
    entries = json.load(open(cache))
    assert len(entries) == 1
    (key, val), = entries.items()
    assert "u16" in key and val["front_words"] == t["front_words"] and val["ms"] > 0
    _check_batch(rx, xs, CFG16)
    # a second context finds the entry and applies it without timing
    r2 = roix.Roix(0)
    try:
        t0 = time.perf_counter()
        t2 = r2.tune(xs, reps=50, cache=cache, **CFG16)
        assert time.perf_counter() - t0 < 1.0
        assert t2 == t
    finally:
        r2.close()
    # another shape class gets an entry of its own
    x = phantom.porous_cylinder(96, radius=36, seed=6, device="cuda")
    rx.tune([x], reps=3, cache=cache, **CFG32)
    assert len(json.load(open(cache))) == 2
    _check_batch(rx, [x], CFG32)
