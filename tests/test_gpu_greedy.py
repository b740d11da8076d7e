"""The 8-bit preprocessor path on the GPU against the oracle: normalisation
(Sec. 4.1.2), uint8 thresholding and compaction, and the greedy quantiser
(Sec. 4.2.3). Every output is integer: compared bit for bit."""
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


def _pack(mask: np.ndarray) -> torch.Tensor:
    """0/1 array (z, y, x) -> mask words (rows x ceil(nx/32), bit x%32 of word x/32)."""
    nx = mask.shape[-1]
    W = (nx + 31) // 32
    m = np.zeros((mask.size // nx, W * 32), np.uint8)
    m[:, :nx] = mask.reshape(-1, nx)
    words = np.packbits(m, axis=1, bitorder="little").view("<u4")
    return torch.from_numpy(words.reshape(-1).astype(np.int64).astype(np.uint32).view(np.int32)).cuda()


NORM_CASES = [
    ("f32_ellipsoids", lambda: phantom.ellipsoids(48, seed=1).numpy(), 0),
    ("f32_ragged", lambda: phantom.ellipsoids(shape=(7, 13, 37), seed=2).numpy(), 0),
    ("f32_specials", lambda: np.array([0, -1, np.nan, np.inf, -np.inf, 3.5, 7.0, 1e-30, 6.99999],
                                      np.float32), 0),
    ("f32_zero", lambda: np.zeros((3, 5, 17), np.float32), 0),
    ("u16_projection", lambda: phantom.projection(512, 3, seed=0).numpy(), 100),
    ("u16_ragged", lambda: phantom.projection(512, 4, seed=1).numpy()[:301, :333], 100),
    ("u16_dark_above", lambda: np.full((4, 40), 50, np.uint16), 60),
    ("f32_tail", lambda: phantom.random_field((1, 997, 1003), seed=3), 0),
]


@pytest.mark.parametrize("name,make,dark", NORM_CASES, ids=[c[0] for c in NORM_CASES])
def test_normalize8_matches_oracle(rx, name, make, dark):
    x = np.ascontiguousarray(make())
    want, imax = oracle.normalize8(x, dark=dark)
    got, gmax = rx.normalize8(torch.from_numpy(x).cuda(), dark=dark)
    rx.sync()
    assert float(gmax.item()) == imax
    assert np.array_equal(got.cpu().numpy(), want)


def test_normalize8_misaligned_views(rx):
    x = phantom.ellipsoids(40, seed=5).numpy().reshape(-1)
    xd = torch.from_numpy(x).cuda()
    for off in (1, 2, 3):
        sub = xd[off:off + 40000]
        want, _ = oracle.normalize8(x[off:off + 40000])
        out = torch.empty(40000 + 1, dtype=torch.uint8, device="cuda")[1:]
        got, _ = rx.normalize8(sub, out=out)
        rx.sync()
        assert np.array_equal(got.cpu().numpy(), want)


U8_ROI = [
    ("gt_dilate", (6, 21, 70), dict(threshold=120, cmp="gt", dilate=1)),
    ("lt_nodilate", (3, 40, 96), dict(threshold=60, cmp="lt", dilate=0)),
    ("keep26", (12, 20, 48), dict(threshold=140, cmp="gt", dilate=1, keep="largest")),
    ("wide_vec", (2, 9, 2048), dict(threshold=100, cmp="gt", dilate=1)),
]


@pytest.mark.parametrize("name,shape,cfg", U8_ROI, ids=[c[0] for c in U8_ROI])
def test_uint8_roi_and_compaction(rx, name, shape, cfg):
    img = phantom.walk8(shape, seed=7, step=6)
    x = torch.from_numpy(img).cuda()
    D = oracle.mask(img, **cfg)
    words, pop = rx.extract_roi(x, **cfg)
    rx.sync()
    nz, ny, nx = shape
    W = (nx + 31) // 32
    bits = np.unpackbits(words.cpu().numpy().view(np.uint8), bitorder="little")
    got = bits.reshape(ny * nz, W * 32)[:, :nx].reshape(shape)
    assert np.array_equal(got, D) and int(pop.item()) == int(D.sum())
    P, counts, bounds = oracle.compact(img, D)
    gp, gc, gb, sizes = rx.compact(x, words)
    rx.sync()
    n, nb = (int(v) for v in sizes.cpu().numpy())
    assert n == P.size and nb == bounds.size
    assert np.array_equal(gp[:n].cpu().numpy(), P)
    assert np.array_equal(gc.cpu().numpy(), counts)
    assert np.array_equal(gb[:nb].cpu().numpy(), bounds)


GREEDY_CASES = [
    # (name, shape, mask density, mean run, step, eabs values)
    ("ragged_multiwin", (3, 37, 301), 0.7, 90.0, 2, (0, 0.6, 1, 2.5, 7, 40, 300)),
    ("long_rows", (1, 40, 4000), 0.9, 900.0, 1, (1, 3, 10)),
    ("short_runs", (2, 70, 130), 0.4, 3.0, 8, (0, 2, 5)),
    ("flat", (1, 33, 700), 1.0, 1e9, 0, (0, 1)),
    ("nx1", (5, 50, 1), 0.5, 1.0, 5, (1,)),
    ("many_rows", (64, 64, 72), 0.5, 20.0, 4, (2,)),
]


@pytest.mark.parametrize("name,shape,density,mean_run,step,ebs", GREEDY_CASES,
                         ids=[c[0] for c in GREEDY_CASES])
def test_greedy_matches_oracle(rx, name, shape, density, mean_run, step, ebs):
    img = phantom.walk8(shape, seed=11, step=step)
    D = phantom.runs(shape, seed=12, density=density, mean_run=mean_run)
    P, _, _ = oracle.compact(img, D)
    words = _pack(D)
    pd = torch.from_numpy(P.copy() if P.size else np.zeros(1, np.uint8)).cuda()
    for e in ebs:
        want = oracle.greedy_rows(img, D, e)
        got, n = rx.greedy(pd, words, shape, e)
        rx.sync()
        assert int(n.item()) == P.size
        assert np.array_equal(got[:P.size].cpu().numpy(), want), f"eabs={e}"
        assert (np.abs(want.astype(int) - P.astype(int)) <= int(np.floor(e))).all()


def test_greedy_in_place_and_empty(rx):
    shape = (4, 33, 257)
    img = phantom.walk8(shape, seed=13, step=3)
    D = phantom.runs(shape, seed=14, density=0.6, mean_run=50.0)
    P, _, _ = oracle.compact(img, D)
    buf = torch.from_numpy(P).cuda()
    want = oracle.greedy_rows(img, D, 2)
    got, n = rx.greedy(buf, _pack(D), shape, 2, out=buf)
    rx.sync()
    assert got.data_ptr() == buf.data_ptr()
    assert np.array_equal(buf.cpu().numpy(), want)
    # an empty mask: nothing to write, n = 0
    Z = np.zeros(shape, np.uint8)
    got, n = rx.greedy(torch.zeros(8, dtype=torch.uint8, device="cuda"), _pack(Z), shape, 2)
    rx.sync()
    assert int(n.item()) == 0


def test_greedy_batch_matches_oracle(rx):
    shapes = [(1, 64, 512), (3, 37, 301), (1, 1, 5), (2, 0, 40), (1, 200, 2048), (1, 31, 70)]
    items, wants, Ps = [], [], []
    for k, shape in enumerate(shapes):
        img = phantom.walk8(shape, seed=20 + k, step=3)
        D = phantom.runs(shape, seed=40 + k, density=0.6, mean_run=60.0)
        P, _, _ = oracle.compact(img, D)
        Ps.append(P)
        wants.append(oracle.greedy_rows(img, D, 2))
        items.append((torch.from_numpy(P if P.size else np.zeros(1, np.uint8)).cuda(),
                      _pack(D) if D.size else torch.zeros(1, dtype=torch.int32, device="cuda"),
                      shape))
    outs, n = rx.greedy_batch(items, 2)
    rx.sync()
    for q, c, w in zip(outs, n.cpu().numpy(), wants):
        assert int(c) == w.size and np.array_equal(q[:w.size].cpu().numpy(), w)


def test_greedy_rejects_bad_arguments(rx):
    import paper_2602_15917_gb300 as roix
    shape = (1, 2, 40)
    words = _pack(np.ones(shape, np.uint8))
    p = torch.zeros(80, dtype=torch.uint8, device="cuda")
    for e in (-1.0, float("nan"), float("inf")):
        with pytest.raises(roix.RoixError):
            rx.greedy(p, words, shape, e)


def test_uint8_refused_by_the_coder(rx):
    import paper_2602_15917_gb300 as roix
    x = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(roix.RoixError):
        rx.compress_bytes(x)


def _chain_oracle(x, dark, roi, eabs):
    img, _ = oracle.normalize8(x, dark=dark)
    D = oracle.mask(img, **roi)
    P, counts, bounds = oracle.compact(img, D)
    return img, D, counts, bounds, oracle.greedy_rows(img, D, eabs)


def _chain_gpu(rx, xd, dark, roi, eabs):
    img, _ = rx.normalize8(xd, dark=dark)
    words, pop = rx.extract_roi(img, **roi)
    P, counts, bounds, sizes = rx.compact(img, words)
    Q, n = rx.greedy(P, words, img.shape, eabs)
    rx.sync()
    return img, words, counts, bounds, sizes, Q, n


@pytest.mark.parametrize("eabs", [1, 4])
def test_paper_chain_projection(rx, eabs):
    """raw projection -> I_n -> threshold on I_n -> compaction -> greedy."""
    x = phantom.projection(1024, 5, seed=2).numpy()
    roi = dict(threshold=200, cmp="lt", dilate=0)
    img, D, counts, bounds, want = _chain_oracle(x, 100, roi, eabs)
    gimg, words, gc, gb, sizes, Q, n = _chain_gpu(rx, torch.from_numpy(x).cuda(), 100, roi, eabs)
    assert np.array_equal(gimg.cpu().numpy(), img)
    assert np.array_equal(gc.cpu().numpy(), counts)
    nn = int(n.item())
    assert nn == want.size == int(sizes[0].item())
    assert np.array_equal(Q[:nn].cpu().numpy(), want)


def test_paper_chain_volume(rx):
    x = phantom.porous_cylinder(160, radius=60.0, seed=3).numpy()
    roi = dict(threshold=25, cmp="gt", dilate=1)
    img, D, counts, bounds, want = _chain_oracle(x, 0, roi, 3)
    gimg, words, gc, gb, sizes, Q, n = _chain_gpu(rx, torch.from_numpy(x).cuda(), 0, roi, 3)
    nn = int(n.item())
    assert np.array_equal(gimg.cpu().numpy(), img)
    assert nn == want.size and np.array_equal(Q[:nn].cpu().numpy(), want)
