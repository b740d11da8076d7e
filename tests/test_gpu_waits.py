"""Bounded device waits end in ROIX_ETIMEOUT, never in a hung GPU.

The tile scans (compaction and pack offsets) and the decoder's row scans wait
on the prefix of the tile before them. The test hook roix_debug_hold_scans
leaves the first tile's prefix unpublished (a flag that nothing sets), and a
short wait limit (roix_set_wait_limit, 1000 polls) makes the next tile give
up. The launch must end, roix_sync must report ROIX_ETIMEOUT, and the next
call on the same context must give the oracle's bytes again.
"""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
import phantom

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    r = roix.Roix(0)
    yield r
    r.close()


def _expect_timeout(rx):
    import paper_2602_15917_gb300 as roix
    t0 = time.perf_counter()
    with pytest.raises(roix.RoixError) as ei:
        rx.sync()
    assert ei.value.status == ETIMEOUT
    assert time.perf_counter() - t0 < 30.0


def _held_then_released(rx, x: np.ndarray, tuning=None, **cfg):
    default = rx.get_tuning()
    try:
        if tuning:
            rx.set_tuning(**tuning)
        xd = torch.from_numpy(x).cuda()
        ref = oracle.compress(x, **cfg)
        rx.set_wait_limit(1000)
        rx.debug_hold_scans(True)
        rx.compress(xd, **cfg)
        _expect_timeout(rx)
        # the same context, hook off and the default limit (1000 polls is too
        # short for a scan tile that waits on a busy predecessor): the oracle's
        # container again
        rx.debug_hold_scans(False)
        rx.set_wait_limit(0)
        got = rx.compress_bytes(xd, **cfg).cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref)
        # decoder row scans (more than one 1024-row tile)
        buf = torch.from_numpy(ref).cuda()
        rx.set_wait_limit(1000)
        rx.debug_hold_scans(True)
        rx.decode(buf, x.shape, torch.from_numpy(x[:0]).dtype)
        _expect_timeout(rx)
        rx.debug_hold_scans(False)
        rx.set_wait_limit(0)
        y = rx.decode(buf, x.shape, torch.from_numpy(x[:0]).dtype)
        rx.sync()
        y_ref = oracle.decode(ref, x.shape, x.dtype)
        assert np.array_equal(y.cpu().numpy().view(np.uint8), y_ref.view(np.uint8))
    finally:
        rx.debug_hold_scans(False)
        rx.set_wait_limit(0)
        rx.set_tuning(**default)


def test_pack_scan_wait_times_out_then_context_recovers(rx):
    # 2.3 M retained values in chunks of 256: 8985 pack chunks, two scan tiles
    x = phantom.random_field((1, 1123, 2048), seed=41)
    cfg = dict(eb=1e-3, eb_mode="abs", threshold=-1e30, dilate=0, chunk=256, radius=64)
    assert (x.size + 255) // 256 > 8192
    _held_then_released(rx, x, **cfg)


def test_compaction_scan_wait_times_out_then_context_recovers(rx):
    # one mask row (256 words) per compaction tile: 8200 tiles, two scan tiles
    rng = np.random.default_rng(42)
    x = rng.integers(90, 4000, (1, 8200, 8192), dtype=np.uint16)
    cfg = dict(eb=4, eb_mode="abs", cmp="lt", threshold=3000, dark=0, dilate=0, fill=0)
    _held_then_released(rx, x, tuning=dict(front_words=256), **cfg)
