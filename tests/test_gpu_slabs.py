"""z-slab compression (roix_compress_slabs) against the oracle, through the C ABI.

A volume cut into z-slabs keeps the whole volume's mask (the dilation crosses
slab borders) and error bound (a relative bound takes the range of every
retained value), with one container per slab. Every container must equal the
oracle's (oracle.compress_slabs) byte for byte, and the GPU decoder must give
the oracle's decode of each slab bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    r = roix.Roix(0)
    yield r
    r.close()


def _run(rx, x: np.ndarray, slab_z: int, **cfg):
    xt = torch.from_numpy(x).cuda()
    outs, sizes = rx.compress_slabs(xt, slab_z, **cfg)
    rx.sync()
    return [o[:int(s)].cpu().numpy() for o, s in zip(outs, sizes.cpu().numpy())]


def _same(ref, got):
    assert len(ref) == len(got)
    for k, (a, b) in enumerate(zip(ref, got)):
        assert a.size == b.size, (k, a.size, b.size)
        if not np.array_equal(a, b):
            i = int(np.nonzero(a != b)[0][0])
            raise AssertionError(f"slab {k}: first differing byte {i} of {a.size}")


CFGS = [dict(eb=1e-3, eb_mode="abs", dilate=1),
        dict(eb=1e-3, eb_mode="rel", dilate=1),
        dict(eb=1e-2, eb_mode="rel", dilate=0),
        dict(eb=1e-4, eb_mode="rel", dilate=1, radius=64, chunk=256, fill=0.25)]


@pytest.mark.parametrize("ci", range(len(CFGS)))
@pytest.mark.parametrize("slab_z", [1, 4, 7, 23, 40])
def test_slabs_equal_oracle(rx, ci, slab_z):
    cfg = CFGS[ci]
    x = phantom.ellipsoids(shape=(23, 18, 21), seed=8).numpy()
    _same(oracle.compress_slabs(x, slab_z, **cfg), _run(rx, x, slab_z, **cfg))


@pytest.fixture(params=[0, 1], ids=["front_blk", "front_warp"])
def front_kernel(rx, request):
    # both compaction counting kernels: the dilation reads the neighbouring
    # slabs' mask planes in each (the autotuner may pick either)
    default = rx.get_tuning()
    rx.set_tuning(front_kernel=request.param)
    yield request.param
    rx.set_tuning(**default)


@pytest.mark.parametrize("shape,slab_z", [((40, 33, 100), 16), ((17, 64, 32), 5),
                                          ((9, 70, 1), 2), ((130, 20, 45), 64),
                                          ((12, 9, 1100), 5)])
def test_slabs_ragged_shapes(rx, front_kernel, shape, slab_z):
    cfg = dict(eb=1e-4, eb_mode="rel", dilate=1)
    if max(shape) <= 130:
        x = phantom.porous_cylinder(max(shape), radius=max(shape) * 0.35, seed=3).numpy()
        x = np.ascontiguousarray(x[:shape[0], :shape[1], :shape[2]])
    else:  # rows of more than 32 mask words, many short runs across the slab borders
        x = np.random.default_rng(3).random(shape, dtype=np.float32)
        cfg["threshold"] = 0.98
    _same(oracle.compress_slabs(x, slab_z, **cfg), _run(rx, x, slab_z, **cfg))


def test_slabs_textured_cylinder_sweep(rx, front_kernel):
    # the 2048^3 workload's phantom at 96^3, 16-slice slabs, the eb sweep
    x = phantom.porous_cylinder(96, radius=37.5, texture=True, seed=1).numpy()
    for eb in (1e-2, 1e-3, 1e-4, 1e-5):
        cfg = dict(eb=eb, eb_mode="rel", dilate=1)
        _same(oracle.compress_slabs(x, 16, **cfg), _run(rx, x, 16, **cfg))


def test_slabs_uint16(rx):
    x = np.stack([phantom.projection(120, i, seed=6).numpy() for i in range(10)])
    for cfg in (dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=1, fill=60100),
                dict(eb=0, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100),
                dict(eb=1e-3, eb_mode="rel", cmp="lt", threshold=57000, dark=100, dilate=1)):
        _same(oracle.compress_slabs(x, 3, **cfg), _run(rx, x, 3, **cfg))


def test_slabs_special_values_and_empty(rx):
    x = phantom.ellipsoids(shape=(12, 16, 40), seed=9).numpy()
    x[3, 5, 7:12] = [np.nan, np.inf, -np.inf, 3e38, 1e-42]
    for cfg in (dict(eb=1e-3, eb_mode="rel"), dict(eb=1e-3, threshold=1e30),
                dict(eb=1e-3, threshold=-1e30)):
        _same(oracle.compress_slabs(x, 5, **cfg), _run(rx, x, 5, **cfg))


def test_one_slab_is_the_plain_container(rx):
    x = phantom.ellipsoids(shape=(20, 24, 36), seed=10).numpy()
    cfg = dict(eb=1e-3, eb_mode="rel", dilate=1)
    got = _run(rx, x, 20, **cfg)
    assert len(got) == 1
    assert np.array_equal(got[0], rx.compress_bytes(torch.from_numpy(x).cuda(), **cfg)
                          .cpu().numpy())


def test_slab_decodes_match_oracle(rx):
    x = phantom.porous_cylinder(64, radius=24, texture=True, seed=2).numpy()
    cfg = dict(eb=1e-4, eb_mode="rel", dilate=1, fill=0.0)
    got = _run(rx, x, 10, **cfg)
    whole = oracle.decode(oracle.compress(x, **cfg), x.shape, np.float32)
    parts = []
    for c in got:
        h = oracle.header(c)
        shape = (h["nz"], h["ny"], h["nx"])
        y = rx.decode(torch.from_numpy(c).cuda(), shape, torch.float32)
        rx.sync()
        a = y.cpu().numpy()
        assert np.array_equal(a.view(np.uint32), oracle.decode(c, shape, np.float32)
                              .view(np.uint32))
        parts.append(a)
    # stacked, the slab decodes are the whole-volume decode
    assert np.array_equal(np.concatenate(parts).view(np.uint32), whole.view(np.uint32))


def test_slabs_refused_arguments(rx):
    import paper_2602_15917_gb300 as roix
    x = torch.from_numpy(phantom.ellipsoids(16, seed=1).numpy()).cuda()
    with pytest.raises(roix.RoixError) as ei:
        rx.compress_slabs(x, 4, keep="largest")
    assert ei.value.status == 1
    with pytest.raises(roix.RoixError):
        rx.compress_slabs(x, 0)
    # the context stays usable
    rx.compress_slabs(x, 4, eb=1e-3)
    rx.sync()


def test_slabs_capacity_reports_sizes(rx):
    import paper_2602_15917_gb300 as roix
    x = phantom.ellipsoids(shape=(12, 32, 32), seed=11).numpy()
    cfg = dict(eb=1e-5, eb_mode="abs")
    ref = oracle.compress_slabs(x, 4, **cfg)
    xt = torch.from_numpy(x).cuda()
    outs = [torch.empty(512, dtype=torch.uint8, device="cuda") for _ in ref]
    _, sizes = rx.compress_slabs(xt, 4, outs=outs, **cfg)
    with pytest.raises(roix.RoixError) as ei:
        rx.sync()
    assert ei.value.status == 3
    assert [int(v) for v in sizes.cpu().numpy()] == [r.size for r in ref]
