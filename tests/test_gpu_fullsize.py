"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (batched call, device-resident inputs), under both compaction counting
kernels (the autotuner may pick either).

* 64 uint16 projections (512^2 .. 2048^2): every container equals the
  oracle's, byte for byte.
* 1024^3 float32 porous cylinder, relative bound 1e-4: the whole container
  equals the oracle's byte for byte (the oracle runs once, ~40 s on one host
  core); besides, on every voxel the decoded values lie within E_abs of the
  input on retained voxels and equal the fill elsewhere, and the retained set
  equals threshold + 3x3x3 dilation recomputed with torch.max_pool3d.
* 2048^3 float32 textured cylinder in 64-slice z-slabs (32 GiB in HBM): the
  first, a middle and the last slab's containers equal the oracle's, each
  encoded by the oracle from the slab's slices plus a one-slice halo with the
  whole volume's error bound; every slab by properties.
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


@pytest.fixture(params=[0, 1], ids=["front_blk", "front_warp"])
def front_kernel(rx, request):
    # both compaction counting kernels (the autotuner may pick either)
    default = rx.get_tuning()
    rx.set_tuning(front_kernel=request.param)
    yield request.param
    rx.set_tuning(**default)


def test_projections64_batch_equals_oracle(rx, front_kernel):
    cfg = dict(eb=4, eb_mode="abs", cmp="lt", threshold=57000, dark=100, dilate=0,
               fill=60100, radius=512, chunk=4096)
    xs = [phantom.projection(s, i, seed=0, device="cuda")
          for i, s in enumerate(phantom.projection_sides(64, 512, 2048, 0))]
    outs, sizes = rx.compress_batch(xs, **cfg)
    rx.sync()
    for x, o, sz in zip(xs, outs, sizes.cpu().numpy()):
        ref = oracle.compress(x.cpu().numpy(), **cfg)
        got = o[:int(sz)].cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref)


def _row_from_container(buf: np.ndarray, hdr: dict, row: int):
    counts = np.frombuffer(buf[hdr["off_counts"]:hdr["off_counts"] + 2 * (hdr["ny"] * hdr["nz"])],
                           np.uint16)
    b0 = int(counts[:row].astype(np.int64).sum())
    return buf[hdr["off_bounds"] + 2 * b0: hdr["off_bounds"] + 2 * (b0 + int(counts[row]))].view(
        np.uint16)


CUBE_CFG = dict(eb=1e-4, eb_mode="rel", cmp="gt", threshold=0.1, dilate=1, fill=0.0,
                radius=512, chunk=4096)


@pytest.fixture(scope="module")
def cube1024(rx):
    """The 1024^3 volume on the device and the oracle's container of it."""
    x = phantom.porous_cylinder(1024, radius=400.0, seed=0, device="cuda")
    ref = oracle.compress(x.cpu().numpy(), **CUBE_CFG)
    yield x, ref
    del x
    torch.cuda.empty_cache()


def test_cube1024_container_equals_oracle(rx, front_kernel, cube1024):
    x, ref = cube1024
    cfg = CUBE_CFG
    outs, sizes = rx.compress_batch([x], **cfg)
    rx.sync()
    buf_d = outs[0][:int(sizes[0].item())]
    buf = buf_d.cpu().numpy()
    # (c) the whole container, byte for byte
    assert buf.size == ref.size
    if not np.array_equal(buf, ref):
        bad = np.flatnonzero(buf != ref)
        raise AssertionError(f"{bad.size} bytes differ, first at {bad[0]} of {buf.size}")
    hdr = oracle.header(buf)
    y = rx.decode(buf_d, x.shape, torch.float32)
    rx.sync()
    # (a) properties on every voxel
    T = (x > 0.1).float()[None, None]
    D = torch.nn.functional.max_pool3d(T, 3, stride=1, padding=1)[0, 0] > 0
    del T
    assert int(D.sum().item()) == hdr["n"]
    eb = hdr["eb_abs"]
    finite = torch.isfinite(x)
    xr, yr = x[D & finite].double(), y[D & finite].double()
    assert float((xr - yr).abs().max().item()) <= eb
    del xr, yr
    assert bool((y[~D] == 0).all().item())
    # the range the relative bound was taken from
    assert hdr["vmin"] == float(x[D].min().item()) and hdr["vmax"] == float(x[D].max().item())


def test_cube2048_slabs_containers_and_properties():
    """2048^3 float32 textured porous cylinder (32 GiB in HBM), 64-slice
    z-slabs, relative bound 1e-4, in the launch configuration bench.py times.
    Per slab, on every voxel: retained count = popcount of threshold + 3x3x3
    dilation (recomputed by torch with a one-slice halo from the neighbouring
    slabs), decoded values within E_abs of the input on retained voxels and the
    fill elsewhere; the whole-volume range and the E_abs constants derived from
    it by the oracle are in every header; sampled rows are recomputed by the
    oracle from their 3x3 neighbourhood of input rows; the first, a middle and
    the last slab's containers equal the oracle's byte for byte."""
    import paper_2602_15917_gb300 as roix
    free, _ = torch.cuda.mem_get_info()
    if free < 140 << 30:
        pytest.skip("needs about 140 GB of free device memory")
    n, slab = 2048, 64
    cfg = dict(eb=1e-4, eb_mode="rel", cmp="gt", threshold=0.1, dilate=1, fill=0.0,
               radius=512, chunk=4096)
    x = phantom.porous_cylinder(n, radius=800.0, texture=True, seed=0, device="cuda")
    rx = roix.Roix(0)
    ns = n // slab
    cap = slab * n * n * 4 // 4
    outs = [torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(ns)]
    rx.reserve(rx.slabs_workspace_size(x.shape, slab, cap=cap, **cfg))
    outs, sizes = rx.compress_slabs(x, slab, outs=outs, **cfg)
    rx.sync()
    sizes = [int(v) for v in sizes.cpu().numpy()]
    hdrs = [oracle.header(o[:256].cpu().numpy()) for o in outs]
    # whole-volume range of the retained values, slab by slab
    vmin, vmax, Ds = float("inf"), float("-inf"), []
    for k in range(ns):
        z0, z1 = k * slab, (k + 1) * slab
        h0, h1 = max(0, z0 - 1), min(n, z1 + 1)
        T = (x[h0:h1] > 0.1).float()[None, None]
        D = torch.nn.functional.max_pool3d(T, 3, stride=1, padding=1)[0, 0, z0 - h0:z0 - h0 + slab] > 0
        del T
        assert int(D.sum().item()) == hdrs[k]["n"], k
        if hdrs[k]["n"]:
            xs_ = x[z0:z1][D]
            xs_ = xs_[torch.isfinite(xs_)]
            vmin = min(vmin, float(xs_.min().item()))
            vmax = max(vmax, float(xs_.max().item()))
            del xs_
        Ds.append(D.cpu())
        del D
    e = oracle.error_bound(np.array([vmin, vmax], np.float32), "rel", cfg["eb"])
    for h in hdrs:
        assert h["vmin"] == vmin and h["vmax"] == vmax
        assert (h["eb_abs"], h["two_eb"], h["inv2eb"], h["bound"]) == \
            (e.eb_abs, np.float32(e.two_eb), np.float32(e.inv2eb), np.float32(e.bound))
    # decoded values, slab by slab
    for k in range(ns):
        z0 = k * slab
        y = rx.decode(outs[k][:sizes[k]], (slab, n, n), torch.float32)
        rx.sync()
        D = Ds[k].cuda()
        xk = x[z0:z0 + slab]
        fin = D & torch.isfinite(xk)
        if bool(fin.any().item()):
            assert float((xk[fin].double() - y[fin].double()).abs().max().item()) <= e.eb_abs
        assert bool((y[~D] == 0).all().item())
        del y, D, fin
    # sampled rows against the oracle
    rng = np.random.default_rng(7)
    zs = rng.integers(590, 1458, 24)
    zs[:6] = [0, 63, 64, 597, 1023, 2047]
    ys = rng.integers(0, n, 24)
    for z, yy in zip(zs.tolist(), ys.tolist()):
        k = z // slab
        buf = outs[k][:sizes[k]].cpu().numpy()
        z0, z1 = max(0, z - 1), min(n, z + 2)
        y0, y1 = max(0, yy - 1), min(n, yy + 2)
        block = x[z0:z1, y0:y1].cpu().numpy()
        Dm = oracle.mask(block, **cfg)[z - z0, yy - y0]
        row = x[z:z + 1, yy:yy + 1].cpu().numpy()
        P, counts, bounds = oracle.compact(row, Dm[None, None])
        assert np.array_equal(_row_from_container(buf, hdrs[k], (z - k * slab) * n + yy), bounds)
        q, o = oracle.quantize(P, e)
        want = np.where(o.astype(bool), P, (q.astype(np.float32) * np.float32(e.two_eb)))
        got = rx.decode(outs[k][:sizes[k]], (slab, n, n), torch.float32)[z - k * slab, yy]
        rx.sync()
        assert np.array_equal(got.cpu().numpy()[Dm.astype(bool)].view(np.uint32),
                              want.astype(np.float32).view(np.uint32))
    # first, middle and last slab: the whole container against the oracle's,
    # encoded from the slab's slices and a one-slice halo with the volume's bound
    for k in (0, ns // 2, ns - 1):
        z0 = k * slab
        h0, h1 = max(0, z0 - 1), min(n, z0 + slab + 1)
        ref = oracle.encode_slab(x[h0:h1].cpu().numpy(), z0 - h0, slab, e, **cfg)
        got = outs[k][:sizes[k]].cpu().numpy()
        assert got.size == ref.size, k
        assert np.array_equal(got, ref), k
    rx.close()
    del x, outs
    torch.cuda.empty_cache()
