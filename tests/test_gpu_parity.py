"""CUDA path against the CPU oracle, through the C ABI, on seeded inputs.

Integer outputs (masks, geometry, codes, symbols, container bytes) must be
bit-identical; decoded values must be bit-identical to the oracle's decode
(the error bound itself is pinned on the oracle side)."""
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


def _unpack_mask(words: torch.Tensor, shape) -> np.ndarray:
    nz, ny, nx = shape
    W = (nx + 31) // 32
    w = words.cpu().numpy().view(np.uint32).reshape(ny * nz, W)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(ny * nz, W * 32)
    return bits[:, :nx].reshape(shape).astype(np.uint8)


def _compress_both(rx, x: np.ndarray, **cfg):
    ref = oracle.compress(x, **cfg)
    got = rx.compress_bytes(torch.from_numpy(x).cuda(), **cfg).cpu().numpy()
    return ref, got


def _assert_same_container(ref, got):
    if got.size != ref.size or not np.array_equal(got, ref):
        h_r, h_g = oracle.header(ref), oracle.header(got) if got.size >= 256 else {}
        diff = {k: (h_r[k], h_g.get(k)) for k in h_r if h_r[k] != h_g.get(k)}
        first = int(np.flatnonzero(got[:min(got.size, ref.size)] != ref[:min(got.size, ref.size)])[0]) \
            if min(got.size, ref.size) and (got[:min(got.size, ref.size)] != ref[:min(got.size, ref.size)]).any() else -1
        raise AssertionError(f"containers differ: sizes {got.size} vs {ref.size}, "
                             f"header diff {diff}, first differing byte {first}")


F32_CASES = [
    ("ellipsoids48", lambda: phantom.ellipsoids(48, seed=1).numpy(), {}),
    ("ragged", lambda: phantom.ellipsoids(shape=(17, 23, 33), seed=2).numpy(), {}),
    ("wide_rows", lambda: phantom.ellipsoids(shape=(5, 7, 100), seed=3).numpy(), {}),
    ("nx32", lambda: phantom.ellipsoids(shape=(9, 11, 32), seed=4).numpy(), {}),
    ("nx64_2d", lambda: phantom.ellipsoids(shape=(1, 64, 64), seed=5).numpy(), {}),
    ("nx1", lambda: phantom.random_field((3, 50, 1), seed=6), dict(threshold=0.0)),
    ("single", lambda: np.array([[[0.5]]], np.float32), {}),
    ("no_dilate", lambda: phantom.ellipsoids(40, seed=7).numpy(), dict(dilate=0)),
    ("below", lambda: phantom.ellipsoids(40, seed=8).numpy(), dict(cmp="lt", threshold=0.5)),
    ("rel", lambda: phantom.porous_cylinder(40, radius=15, seed=1).numpy(),
     dict(eb=1e-3, eb_mode="rel")),
    ("rel_tight", lambda: phantom.porous_cylinder(40, radius=15, seed=2).numpy(),
     dict(eb=1e-5, eb_mode="rel")),
    ("radius2", lambda: phantom.ellipsoids(32, seed=9).numpy(), dict(radius=2)),
    ("radius2048_chunk256", lambda: phantom.ellipsoids(32, seed=10).numpy(),
     dict(radius=2048, chunk=256, eb=1e-5)),
    ("chunk16384", lambda: phantom.ellipsoids(48, seed=11).numpy(), dict(chunk=16384)),
    ("all_roi", lambda: phantom.random_field((4, 9, 70), seed=12), dict(threshold=-1e30)),
    ("no_roi", lambda: phantom.random_field((4, 9, 70), seed=13), dict(threshold=1e30)),
    ("noise_white", lambda: phantom.random_field((6, 20, 90), seed=14, smooth=False),
     dict(threshold=-0.5, eb=1e-2)),
    ("fill", lambda: phantom.ellipsoids(24, seed=15).numpy(), dict(fill=-7.25)),
]


@pytest.mark.parametrize("name,make,cfg", F32_CASES, ids=[c[0] for c in F32_CASES])
def test_fused_float32_bit_exact(rx, name, make, cfg):
    x = make()
    base = dict(eb=1e-3, eb_mode="abs", threshold=0.1, dilate=1)
    base.update(cfg)
    ref, got = _compress_both(rx, x, **base)
    _assert_same_container(ref, got)


def test_fused_float32_special_values(rx):
    x = phantom.random_field((5, 13, 77), seed=20)
    flat = x.reshape(-1)
    flat[::37] = np.nan
    flat[5::41] = np.inf
    flat[7::43] = -np.inf
    flat[9::47] = 3e38
    flat[11::53] = -1e-41  # subnormal
    flat[13::59] = -0.0
    for eb in (1e-3, 1e-40, 1e30):
        ref, got = _compress_both(rx, x, eb=eb, threshold=-1.0, dilate=1)
        _assert_same_container(ref, got)


def test_fused_config1_workload(rx):
    # 128^3 ellipsoid phantom, eb 1e-3 absolute, threshold 0.1, 1-voxel dilation
    x = phantom.ellipsoids(128, seed=0).numpy()
    ref, got = _compress_both(rx, x, eb=1e-3, threshold=0.1, dilate=1)
    _assert_same_container(ref, got)
    assert got.size < x.nbytes / 2


U16_CASES = [
    ("proj", (200, 211), dict(eb=4)),
    ("proj_lossless", (97, 130), dict(eb=0)),
    ("proj_dilate", (150, 150), dict(eb=4, dilate=1)),
    ("proj_rel", (128, 160), dict(eb=1e-4, eb_mode="rel")),
    ("proj_nx32", (40, 32), dict(eb=2)),
]


@pytest.mark.parametrize("name,shape,cfg", U16_CASES, ids=[c[0] for c in U16_CASES])
def test_fused_uint16_bit_exact(rx, name, shape, cfg):
    side = max(shape)
    x = phantom.projection(side, 3, seed=1).numpy()[:shape[0], :shape[1]].copy()
    base = dict(eb=4, eb_mode="abs", cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    base.update(cfg)
    ref, got = _compress_both(rx, x, **base)
    _assert_same_container(ref, got)


def test_staged_chain_matches_oracle_and_fused(rx):
    x = phantom.ellipsoids(shape=(20, 30, 45), seed=30).numpy()
    cfg = dict(eb=2e-3, eb_mode="rel", threshold=0.1, dilate=1)
    xt = torch.from_numpy(x).cuda()
    # extract_roi
    mask, pop = rx.extract_roi(xt, **cfg)
    D = oracle.mask(x, **cfg)
    rx.sync()
    assert np.array_equal(_unpack_mask(mask, x.shape), D)
    assert int(pop.item()) == int(D.sum())
    # compact
    pixels, counts, bounds, sizes = rx.compact(xt, mask)
    rx.sync()
    P, c_ref, b_ref = oracle.compact(x, D)
    n, nb = (int(v) for v in sizes.cpu().numpy())
    assert n == P.size and nb == b_ref.size
    assert np.array_equal(pixels[:n].cpu().numpy(), P)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    assert np.array_equal(bounds[:nb].cpu().numpy(), b_ref)
    # quantize
    q, ob, info = rx.quantize(pixels, n_cap=x.size, n_dev=sizes[:1], **cfg)
    rx.sync()
    e = oracle.error_bound(P, "rel", cfg["eb"])
    q_ref, o_ref = oracle.quantize(P, e)
    assert np.array_equal(q[:n].cpu().numpy(), q_ref)
    obits = np.unpackbits(ob.cpu().numpy().view(np.uint8), bitorder="little")[:n]
    assert np.array_equal(obits, o_ref)
    inf = np.frombuffer(info.cpu().numpy().tobytes(), dtype=[("eb_abs", "<f8"), ("vmin", "<f8"),
                        ("vmax", "<f8"), ("two", "<f4"), ("inv", "<f4"), ("bound", "<f4"),
                        ("ebi", "<i4")])[0]
    assert inf["eb_abs"] == e.eb_abs and inf["two"] == e.two_eb and inf["bound"] == e.bound
    # encode
    out, size = rx.encode(q, ob, pixels, x.size, sizes, counts, bounds, info, x.shape,
                          torch.float32, **cfg)
    rx.sync()
    got = out[:int(size.item())].cpu().numpy()
    ref = oracle.compress(x, **cfg)
    _assert_same_container(ref, got)
    fused = rx.compress_bytes(xt, **cfg).cpu().numpy()
    assert np.array_equal(fused, got)


# Row widths that are multiples of 32 voxels (the x = nx boundary is carried
# past the last word) with word counts that are not multiples of 32, and
# columns of more than one warp width: every mask pattern the per-row counts
# and offsets must get right, dilated or not, in the fused and staged paths.
WORD_EDGE_SHAPES = [(3, 40, 96), (2, 9, 64), (2, 5, 1056), (1, 7, 2048), (2, 6, 1000), (3, 4, 32)]


@pytest.mark.parametrize("shape", WORD_EDGE_SHAPES, ids=["x".join(map(str, s)) for s in WORD_EDGE_SHAPES])
@pytest.mark.parametrize("dilate", [0, 1])
@pytest.mark.parametrize("front_kernel", [0, 1])
def test_row_widths_at_word_edges(rx, shape, dilate, front_kernel):
    x = phantom.ellipsoids(shape=shape, seed=11).numpy()
    x[:, :, -1] = 1.0  # retained last column: rows end inside the ROI
    x[:, 0, :] = 1.0
    cfg = dict(eb=1e-3, threshold=0.1, dilate=dilate)
    default = rx.get_tuning()
    try:
        rx.set_tuning(front_kernel=front_kernel)
        ref, got = _compress_both(rx, x, **cfg)
        _assert_same_container(ref, got)
        xt = torch.from_numpy(x).cuda()
        mask, _ = rx.extract_roi(xt, **cfg)
        pixels, counts, bounds, sizes = rx.compact(xt, mask)
        rx.sync()
    finally:
        rx.set_tuning(**default)
    P, c_ref, b_ref = oracle.compact(x, oracle.mask(x, **cfg))
    n, nb = (int(v) for v in sizes.cpu().numpy())
    assert n == P.size and nb == b_ref.size
    assert np.array_equal(pixels[:n].cpu().numpy(), P)
    assert np.array_equal(counts.cpu().numpy(), c_ref)
    assert np.array_equal(bounds[:nb].cpu().numpy(), b_ref)


def test_staged_uint16(rx):
    x = phantom.projection(180, 4, seed=2).numpy()
    cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    xt = torch.from_numpy(x).cuda()
    mask, pop = rx.extract_roi(xt, **cfg)
    pixels, counts, bounds, sizes = rx.compact(xt, mask)
    q, ob, info = rx.quantize(pixels, n_cap=x.size, n_dev=sizes[:1], **cfg)
    out, size = rx.encode(q, ob, pixels, x.size, sizes, counts, bounds, info, x.shape,
                          torch.uint16, **cfg)
    rx.sync()
    _assert_same_container(oracle.compress(x, **cfg), out[:int(size.item())].cpu().numpy())


@pytest.mark.parametrize("kind", ["f32", "f32_rel", "u16", "empty", "full"])
def test_decode_bit_exact(rx, kind):
    if kind.startswith("f32"):
        x = phantom.ellipsoids(shape=(21, 34, 50), seed=40).numpy()
        cfg = dict(eb=1e-3, eb_mode="rel" if kind == "f32_rel" else "abs", threshold=0.1,
                   dilate=1, fill=0.5)
        dt = torch.float32
    elif kind == "u16":
        x = phantom.projection(160, 5, seed=3).numpy()
        cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
        dt = torch.uint16
    else:
        x = phantom.random_field((3, 10, 40), seed=41)
        cfg = dict(eb=1e-2, threshold=1e30 if kind == "empty" else -1e30, fill=2.0)
        dt = torch.float32
    ref = oracle.compress(x, **cfg)
    y_ref = oracle.decode(ref, x.shape, x.dtype)
    y = rx.decode(torch.from_numpy(ref).cuda(), x.shape, dt)
    rx.sync()
    a = y.cpu().numpy()
    assert np.array_equal(a.view(np.uint8), y_ref.view(np.uint8))


def test_decode_rejects_corrupt(rx):
    import paper_2602_15917_gb300 as roix
    x = phantom.ellipsoids(24, seed=42).numpy()
    ref = oracle.compress(x, eb=1e-3, threshold=0.1)
    buf = torch.from_numpy(ref).cuda()
    for size, shape in [(100, x.shape), (ref.size - 16, x.shape), (ref.size, (24, 24, 25))]:
        rx.decode(buf, shape, torch.float32, size=size)
        with pytest.raises(roix.RoixError) as ei:
            rx.sync()
        assert ei.value.status == 4
    bad = ref.copy()
    bad[0] = 0
    rx.decode(torch.from_numpy(bad).cuda(), x.shape, torch.float32)
    with pytest.raises(roix.RoixError):
        rx.sync()
    # the context stays usable
    rx.decode(buf, x.shape, torch.float32)
    rx.sync()


def test_capacity_error_reports_size(rx):
    import paper_2602_15917_gb300 as roix
    x = torch.from_numpy(phantom.ellipsoids(32, seed=43).numpy()).cuda()
    out = torch.empty(1024, dtype=torch.uint8, device="cuda")
    _, size = rx.compress(x, out=out, eb=1e-4, threshold=0.1)
    with pytest.raises(roix.RoixError) as ei:
        rx.sync()
    assert ei.value.status == 3
    need = int(size.item())
    ref = oracle.compress(x.cpu().numpy(), eb=1e-4, threshold=0.1)
    assert need == ref.size


def test_deterministic_and_stream_ordered(rx):
    x = torch.from_numpy(phantom.porous_cylinder(64, radius=24, seed=5).numpy()).cuda()
    cfg = dict(eb=1e-4, eb_mode="rel", threshold=0.1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = rx.compress_bytes(x, **cfg).clone()
        b = rx.compress_bytes(x, **cfg).clone()
    s.synchronize()
    assert torch.equal(a, b)


def test_batch_equals_single_and_oracle(rx):
    # uneven uint16 projections, one batched call; every container must be the
    # one compress() writes alone, and the oracle's
    sides = [37, 64, 130, 211, 96, 1, 300, 45]
    xs = [phantom.projection(s, i, seed=7).numpy() for i, s in enumerate(sides)]
    cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    outs, sizes = rx.compress_batch([torch.from_numpy(x).cuda() for x in xs], **cfg)
    rx.sync()
    for x, o, sz in zip(xs, outs, sizes.cpu().numpy()):
        got = o[:int(sz)].cpu().numpy()
        _assert_same_container(oracle.compress(x, **cfg), got)


def test_batch_float32_volumes_and_empty_items(rx):
    shapes = [(9, 17, 33), (1, 1, 1), (12, 40, 64), (3, 5, 7), (20, 20, 20)]
    xs = [phantom.ellipsoids(shape=sh, seed=i + 50).numpy() for i, sh in enumerate(shapes)]
    xs[3][:] = -1.0  # nothing above the threshold
    cfg = dict(eb=1e-3, eb_mode="rel", threshold=0.1, dilate=1)
    outs, sizes = rx.compress_batch([torch.from_numpy(x).cuda() for x in xs], **cfg)
    rx.sync()
    for x, o, sz in zip(xs, outs, sizes.cpu().numpy()):
        _assert_same_container(oracle.compress(x, **cfg), o[:int(sz)].cpu().numpy())


def test_batch_more_items_than_one_group(rx):
    xs = [phantom.projection(40 + (i % 7) * 9, i, seed=8).numpy() for i in range(70)]
    cfg = dict(eb=2, cmp="lt", threshold=57000, dark=100, dilate=1, fill=60100)
    outs, sizes = rx.compress_batch([torch.from_numpy(x).cuda() for x in xs], **cfg)
    rx.sync()
    for i in (0, 31, 63, 64, 69):
        _assert_same_container(oracle.compress(xs[i], **cfg),
                               outs[i][:int(sizes[i].item())].cpu().numpy())


def test_batch_under_cuda_graph(rx):
    xs = [torch.from_numpy(phantom.projection(s, i, seed=9).numpy()).cuda()
          for i, s in enumerate([100, 150, 77])]
    cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    outs, sizes = rx.compress_batch(xs, **cfg)  # sizes the workspace, warms up
    rx.sync()
    ref = [o[:int(s)].clone() for o, s in zip(outs, sizes.cpu().numpy())]
    for o in outs:
        o.zero_()
    sizes.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        rx.compress_batch(xs, outs=outs, sizes=sizes, stream=s, **cfg)
    g.replay()
    torch.cuda.synchronize()
    rx.sync()
    for r, o, sz in zip(ref, outs, sizes.cpu().numpy()):
        assert torch.equal(o[:int(sz)], r)


KEEP_CASES = [
    ((7, 9, 33), 26, 0.0), ((7, 9, 33), 6, 0.0), ((12, 20, 70), 26, 0.3),
    ((12, 20, 70), 6, -0.3), ((1, 50, 64), 26, 0.0), ((1, 50, 64), 6, 0.2),
    ((5, 1, 200), 26, 0.0), ((9, 31, 32), 26, 0.5),
]


@pytest.mark.parametrize("shape,conn,thr", KEEP_CASES,
                         ids=[f"{s}-{c}-{t}" for s, c, t in KEEP_CASES])
def test_keep_largest_mask(rx, shape, conn, thr):
    x = phantom.random_field(shape, seed=sum(shape) + conn, smooth=False)
    cfg = dict(threshold=thr, keep="largest", connectivity=conn, dilate=1)
    mask, pop = rx.extract_roi(torch.from_numpy(x).cuda(), **cfg)
    rx.sync()
    D = oracle.mask(x, **cfg)
    assert np.array_equal(_unpack_mask(mask, shape), D)
    assert int(pop.item()) == int(D.sum())


def test_keep_largest_tie_and_empty(rx):
    x = np.zeros((1, 12, 12), np.float32)
    x[0, 1:3, 1:3] = 1.0
    x[0, 8:10, 8:10] = 1.0  # same size: the first one (smallest index) is kept
    cfg = dict(threshold=0.5, keep="largest", dilate=0)
    mask, _ = rx.extract_roi(torch.from_numpy(x).cuda(), **cfg)
    rx.sync()
    assert np.array_equal(_unpack_mask(mask, x.shape), oracle.mask(x, **cfg))
    e = np.zeros((3, 4, 40), np.float32)
    mask, pop = rx.extract_roi(torch.from_numpy(e).cuda(), **cfg)
    rx.sync()
    assert int(pop.item()) == 0


def test_keep_largest_fused_and_batch(rx):
    xs = [phantom.ellipsoids(shape=(20, 30, 45), seed=60).numpy(),
          phantom.random_field((6, 25, 50), seed=61, smooth=False)]
    cfgs = [dict(eb=1e-3, threshold=0.1, keep="largest", dilate=1),
            dict(eb=1e-2, threshold=0.4, keep="largest", connectivity=6, dilate=1)]
    for x, cfg in zip(xs, cfgs):
        ref, got = _compress_both(rx, x, **cfg)
        _assert_same_container(ref, got)
    cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100, keep="largest")
    ps = [phantom.projection(s, i, seed=10).numpy() for i, s in enumerate([90, 120, 64])]
    outs, sizes = rx.compress_batch([torch.from_numpy(p).cuda() for p in ps], **cfg)
    rx.sync()
    for p, o, sz in zip(ps, outs, sizes.cpu().numpy()):
        _assert_same_container(oracle.compress(p, **cfg), o[:int(sz)].cpu().numpy())


def test_keep_largest_repeatable(rx):
    # many small components near the percolation threshold: every run must
    # land on its final root, call after call
    x = phantom.random_field((10, 40, 90), seed=77, smooth=False)
    cfg = dict(threshold=0.4, keep="largest", connectivity=6, dilate=0)
    D = oracle.mask(x, **cfg)
    xt = torch.from_numpy(x).cuda()
    for _ in range(20):
        mask, pop = rx.extract_roi(xt, **cfg)
        rx.sync()
        assert int(pop.item()) == int(D.sum())
        assert np.array_equal(_unpack_mask(mask, x.shape), D)


# Rows that are not 16-byte aligned, nx >= 256: the binarisation reads the
# volume as one flat array (aligned vectors, mask words by funnel shifts).
FLAT_CASES = [((3, 7, 257), np.float32), ((2, 5, 1023), np.float32), ((1, 9, 1025), np.float32),
              ((4, 3, 333), np.float32), ((1, 1, 300), np.float32), ((2, 6, 300), np.uint16),
              ((1, 11, 511), np.uint16), ((3, 4, 1001), np.uint16), ((2, 5, 2047), np.uint16),
              ((5, 7, 270), np.uint8), ((1, 3, 4097), np.uint8)]


@pytest.mark.parametrize("shape,dt", FLAT_CASES, ids=[f"{s}-{d.__name__}" for s, d in FLAT_CASES])
def test_flat_binarisation_masks(rx, shape, dt):
    rng = np.random.default_rng(sum(shape))
    if dt == np.float32:
        x = rng.standard_normal(shape).astype(np.float32)
        cfgs = [dict(threshold=0.3, dilate=0), dict(threshold=0.3, dilate=1),
                dict(cmp="lt", threshold=-1.0, dilate=0)]
    elif dt == np.uint16:
        x = rng.integers(0, 65536, shape).astype(np.uint16)
        cfgs = [dict(cmp="lt", threshold=30000, dark=100, dilate=0),
                dict(cmp="gt", threshold=60000, dark=0, dilate=1)]
    else:
        x = rng.integers(0, 256, shape).astype(np.uint8)
        cfgs = [dict(threshold=128, dilate=0), dict(cmp="lt", threshold=20, dilate=1)]
    xt = torch.from_numpy(x).cuda()
    for cfg in cfgs:
        words, pop = rx.extract_roi(xt, **cfg)
        rx.sync()
        want = oracle.mask(x, **cfg)
        assert np.array_equal(_unpack_mask(words, x.shape), want), cfg
        assert int(pop.item()) == int(want.sum())


def test_flat_binarisation_in_fused_and_batch(rx):
    xs = [phantom.projection(s, i, seed=7).numpy() for i, s in enumerate([257, 301, 515, 999])]
    cfg = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    for x in xs:
        ref, got = _compress_both(rx, x, **cfg)
        _assert_same_container(ref, got)
    outs, sizes = rx.compress_batch([torch.from_numpy(x).cuda() for x in xs], **cfg)
    rx.sync()
    for x, o, sz in zip(xs, outs, sizes.cpu().numpy()):
        _assert_same_container(oracle.compress(x, **cfg), o[:int(sz)].cpu().numpy())
    x = phantom.ellipsoids(shape=(6, 40, 290), seed=3).numpy()
    ref, got = _compress_both(rx, x, eb=1e-3, eb_mode="rel")
    _assert_same_container(ref, got)


@pytest.mark.parametrize("front_kernel", [0, 1])
def test_scans_over_more_tiles_and_chunks_than_one_block(rx, front_kernel):
    # more than 1024 compaction tiles and pack chunks per item: the per-item
    # scans give every thread a range of several entries
    default = rx.get_tuning()
    try:
        # 8 rows of 1024 voxels per tile: 1200 tiles
        rx.set_tuning(front_words=256, front_kernel=front_kernel)
        x = phantom.porous_cylinder(1024, radius=400.0, seed=3, z_range=(440, 456)).numpy()
        x = np.ascontiguousarray(x[:, 212:812, :])  # 16 x 600 x 1024
        for cfg in (dict(eb=1e-4, eb_mode="rel", dilate=1, chunk=256),
                    dict(eb=1e-5, eb_mode="rel", dilate=0, chunk=256, radius=64)):
            ref, got = _compress_both(rx, x, **cfg)
            _assert_same_container(ref, got)
            h = oracle.header(ref)
            assert h["n_chunks"] > 1024
    finally:
        rx.set_tuning(**default)


# The two-layer Lorenzo (predictor = 2): containers equal the oracle's, the
# decoder inverts it bit for bit.
P2_CASES = [
    ("ellipsoids48", lambda: phantom.ellipsoids(48, seed=21).numpy(), {}),
    ("ragged_rel", lambda: phantom.porous_cylinder(40, radius=15, texture=True, seed=2).numpy(),
     dict(eb=1e-4, eb_mode="rel")),
    ("tight_R2", lambda: phantom.ellipsoids(shape=(9, 20, 33), seed=22).numpy(),
     dict(eb=1e-5, radius=2)),
    ("chunk256", lambda: phantom.ellipsoids(40, seed=23).numpy(), dict(chunk=256, radius=64)),
    ("chunk16384", lambda: phantom.ellipsoids(48, seed=24).numpy(), dict(chunk=16384)),
    ("noise", lambda: phantom.random_field((6, 20, 90), seed=25, smooth=False),
     dict(threshold=-0.5, eb=1e-2)),
    ("all_roi", lambda: phantom.random_field((4, 9, 70), seed=26), dict(threshold=-1e30)),
]


@pytest.mark.parametrize("name,make,cfg", P2_CASES, ids=[c[0] for c in P2_CASES])
def test_predictor2_containers_and_decode(rx, name, make, cfg):
    x = make()
    cfg = dict(cfg, predictor=2)
    ref, got = _compress_both(rx, x, **cfg)
    _assert_same_container(ref, got)
    assert oracle.header(got)["order"] == 2
    y = rx.decode(torch.from_numpy(got).cuda(), x.shape, torch.float32)
    rx.sync()
    assert np.array_equal(y.cpu().numpy().view(np.uint32),
                          oracle.decode(ref, x.shape, np.float32).view(np.uint32))


def test_predictor2_specials_uint16_staged_batch_slabs(rx):
    f = phantom.ellipsoids(shape=(6, 16, 40), seed=27).numpy()
    f[2, 3, 5:10] = [np.nan, np.inf, -np.inf, 3e38, 1e-42]
    cfg = dict(eb=1e-3, threshold=-1e30, predictor=2)
    ref, got = _compress_both(rx, f, **cfg)
    _assert_same_container(ref, got)
    y = rx.decode(torch.from_numpy(got).cuda(), f.shape, torch.float32)
    rx.sync()
    assert np.array_equal(y.cpu().numpy().view(np.uint32),
                          oracle.decode(ref, f.shape, np.float32).view(np.uint32))
    # uint16
    p = phantom.projection(150, 3, seed=9).numpy()
    cu = dict(eb=4, cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100, predictor=2)
    ref, got = _compress_both(rx, p, **cu)
    _assert_same_container(ref, got)
    y = rx.decode(torch.from_numpy(got).cuda(), p.shape, torch.uint16)
    rx.sync()
    assert np.array_equal(y.cpu().numpy(), oracle.decode(ref, p.shape, np.uint16))
    # staged chain (codes first) gives the same bytes
    xt = torch.from_numpy(f).cuda()
    mask, _ = rx.extract_roi(xt, **cfg)
    pixels, counts, bounds, sizes = rx.compact(xt, mask)
    q, ob, info = rx.quantize(pixels, n_cap=f.size, n_dev=sizes[:1], **cfg)
    out, size = rx.encode(q, ob, pixels, f.size, sizes, counts, bounds, info, f.shape,
                          torch.float32, **cfg)
    rx.sync()
    _assert_same_container(oracle.compress(f, **cfg), out[:int(size.item())].cpu().numpy())
    # batch and z-slabs
    xs = [phantom.ellipsoids(shape=(5, 20, 30 + 7 * i), seed=30 + i).numpy() for i in range(3)]
    outs, sz = rx.compress_batch([torch.from_numpy(v).cuda() for v in xs], eb=1e-3, predictor=2)
    rx.sync()
    for v, o, s_ in zip(xs, outs, sz.cpu().numpy()):
        _assert_same_container(oracle.compress(v, eb=1e-3, predictor=2), o[:int(s_)].cpu().numpy())
    v = phantom.porous_cylinder(32, radius=12, seed=5).numpy()
    so, ss = rx.compress_slabs(torch.from_numpy(v).cuda(), 7, eb=1e-4, eb_mode="rel", predictor=2)
    rx.sync()
    for r_, o, s_ in zip(oracle.compress_slabs(v, 7, eb=1e-4, eb_mode="rel", predictor=2), so,
                         ss.cpu().numpy()):
        _assert_same_container(r_, o[:int(s_)].cpu().numpy())
