"""Evaluation metrics on the GPU (Sec. 5.2 ROI quality, Sec. 5.6 SSIM)
against the CPU oracle. Counts are exact and the ratios, computed one IEEE
operation at a time in the same order, are bit-identical; the distance sums
and SSIM are sums of many binary64 terms in another order, compared within
the rounding bound of such sums."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import phantom
from oracle import metrics as M

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    r = roix.Roix(0)
    yield r
    r.close()


def _pack(mask: np.ndarray) -> torch.Tensor:
    nx = mask.shape[-1]
    W = (nx + 31) // 32
    m = np.zeros((mask.size // nx, W * 32), np.uint8)
    m[:, :nx] = np.asarray(mask, np.uint8).reshape(-1, nx)
    words = np.packbits(m, axis=1, bitorder="little").view("<u4").reshape(-1)
    if words.size == 0:
        words = np.zeros(1, np.uint32)
    return torch.from_numpy(words.view(np.int32).copy()).cuda()


def _same(a, b):
    return (math.isnan(a) and math.isnan(b)) or a == b


def _check(rx, A, B, distances=True):
    got = rx.roi_quality(_pack(A), _pack(B), A.shape, distances)
    want = M.roi_metrics(A, B)
    for k in ("tp", "fp", "fn", "tn"):
        assert got[k] == want[k], k
    for k in ("dsc", "iou", "sensitivity", "specificity", "accuracy", "kappa", "auc"):
        assert _same(got[k], want[k]), (k, got[k], want[k])
    if distances:
        n = max(1, int(np.count_nonzero(A)) + int(np.count_nonzero(B)))
        for k in ("sum_ab", "sum_ba", "ahd"):
            if math.isnan(want[k]):
                assert math.isnan(got[k]), k
            else:
                assert got[k] == pytest.approx(want[k], rel=4 * n * EPS, abs=1e-300), k
    return got


SHAPES = [(40, 45), (1, 1, 70), (5, 17, 33), (9, 31, 64), (2, 3, 1000), (24, 24, 24)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("seed", [0, 1])
def test_roi_quality_random_masks(rx, shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.random(shape) < 0.3
    B = rng.random(shape) < 0.25
    _check(rx, A, B)


@pytest.mark.parametrize("m,k,dim", [(10, 1, 2), (16, 3, 2), (8, 5, 3), (12, 2, 3)])
def test_ahd_shifted_cube_closed_form(rx, m, k, dim):
    shape = (m + k + 4,) * dim
    A = np.zeros(shape, bool)
    B = np.zeros(shape, bool)
    sl = tuple(slice(2, 2 + m) for _ in range(dim))
    A[sl] = True
    sh = list(sl)
    sh[-1] = slice(2 + k, 2 + m + k)
    B[tuple(sh)] = True
    got = _check(rx, A, B)
    assert got["ahd"] == pytest.approx(k * (k + 1) / (2 * m), rel=1e-12)


def test_roi_quality_empty_and_identical(rx):
    Z = np.zeros((6, 7, 40), bool)
    A = Z.copy()
    A[2, 3, 5] = True
    _check(rx, Z, A)
    _check(rx, A, Z)
    _check(rx, Z, Z)
    got = _check(rx, A, A)
    assert got["dsc"] == 1.0 and got["ahd"] == 0.0


def test_roi_quality_phantom_masks(rx):
    """Predicted = threshold of a noisy ellipsoid volume, truth = the same
    threshold of the noise-free volume: the Sec. 5.2 setting."""
    x = phantom.ellipsoids(64, seed=4).numpy()
    clean = phantom.ellipsoids(64, sigma=0.0, seed=4).numpy()
    _check(rx, x > 0.25, clean > 0.25)
    _check(rx, (x > 0.25)[30], (clean > 0.3)[30], True)  # one 2D slice


def test_roi_quality_without_distances(rx):
    rng = np.random.default_rng(3)
    A = rng.random((4, 50, 50)) < 0.5
    B = rng.random((4, 50, 50)) < 0.5
    got = _check(rx, A, B, distances=False)
    assert math.isnan(got["ahd"])


SSIM_CASES = [
    ("f32", lambda r: (r.random((3, 40, 57)).astype(np.float32) * 2,), 2.0),
    ("u16", lambda r: (r.integers(0, 60000, (2, 64, 70)).astype(np.uint16),), 65535.0),
    ("u8", lambda r: (r.integers(0, 256, (37, 41)).astype(np.uint8),), 255.0),
]


@pytest.mark.parametrize("name,make,L", SSIM_CASES, ids=[c[0] for c in SSIM_CASES])
def test_ssim_matches_oracle(rx, name, make, L):
    rng = np.random.default_rng(5)
    (x,) = make(rng)
    noise = rng.normal(0, 0.05 * L, x.shape)
    y = np.clip(x.astype(np.float64) + noise, 0, L).astype(x.dtype)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    got = float(rx.ssim(xd, yd, L).item())
    want = M.ssim(x, y, L)
    assert got == pytest.approx(want, abs=1e-10)
    assert float(rx.ssim(xd, xd, L).item()) == pytest.approx(1.0, abs=1e-12)


def test_ssim_small_slices_nan(rx):
    x = torch.zeros((4, 10, 30), dtype=torch.float32, device="cuda")
    assert math.isnan(float(rx.ssim(x, x, 1.0).item()))


def test_ssim_of_reconstructions(rx):
    """Sec. 5.6: the decoded projection against the original with the
    background replaced by the fill value; lossless gives exactly 1."""
    import oracle
    x = phantom.projection(512, 2, seed=1).numpy()
    cfg = dict(eb=0, eb_mode="abs", cmp="lt", threshold=57000, dark=100, dilate=0, fill=60100)
    D = oracle.mask(x, **cfg).astype(bool)
    ref = np.where(D, x, np.uint16(60100)).astype(np.uint16)
    xd = torch.from_numpy(x).cuda()
    buf = rx.compress_bytes(xd, **cfg)
    y = rx.decode(buf, x.shape, torch.uint16)
    rx.sync()
    rd = torch.from_numpy(ref).cuda()
    assert float(rx.ssim(rd, y, 65535.0).item()) == pytest.approx(1.0, abs=1e-12)
    cfg["eb"] = 64
    buf = rx.compress_bytes(xd, **cfg)
    y = rx.decode(buf, x.shape, torch.uint16)
    rx.sync()
    got = float(rx.ssim(rd, y, 65535.0).item())
    assert got < 1.0
    assert got == pytest.approx(M.ssim(ref, y.cpu().numpy(), 65535.0), abs=1e-10)
