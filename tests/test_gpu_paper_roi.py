"""Paper-mode ROI on the GPU (multi-Otsu, holes filled, largest object, one
span per row, every 2D slice) against the oracle: thresholds, mask bits and
pixel counts must be identical."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import phantom
from oracle import paper_roi as PR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    r = roix.Roix(0)
    yield r
    r.close()


def _unpack(words: torch.Tensor, shape) -> np.ndarray:
    nz, ny, nx = (1,) * (3 - len(shape)) + tuple(shape)
    W = (nx + 31) // 32
    w = words.cpu().numpy().view(np.uint32).reshape(ny * nz, W)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(ny * nz, W * 32)
    return bits[:, :nx].reshape(shape).astype(np.uint8)


def _check(rx, img):
    want, thr = PR.paper_mask(img)
    words, pop, gthr = rx.extract_roi_paper(torch.from_numpy(np.ascontiguousarray(img)).cuda())
    rx.sync()
    assert np.array_equal(gthr.cpu().numpy().astype(np.int64), thr)
    got = _unpack(words, img.shape)
    assert np.array_equal(got, want), int((got != want).sum())
    assert int(pop.item()) == int(want.sum())


def _disk_image(n=96, seed=0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[:n, :n]
    r = np.hypot(yy - n / 2, xx - n / 2.2)
    img = np.where(r < n / 3, 190, 25).astype(np.float64)
    img[r < n / 9] = 30                               # a hole
    img[(yy > n - 12) & (xx < 20)] = 120              # a grey block at the edge
    img[5:9, n - 9:n - 5] = 200                       # a bright speck
    img += rng.normal(0, 6, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def test_disk_with_hole(rx):
    _check(rx, _disk_image())


@pytest.mark.parametrize("shape,seed", [((70, 45), 1), ((3, 50, 77), 2), ((1, 129), 3),
                                        ((40, 33), 4)])
def test_random_walk_images(rx, shape, seed):
    _check(rx, phantom.walk8(shape, seed=seed, step=9, hold=0.2))


def test_projection_after_normalisation(rx):
    x = phantom.projection(512, 1, seed=0).numpy()
    img, _ = oracle.normalize8(x, dark=100)
    _check(rx, img)


def test_volume_slices(rx):
    x = phantom.porous_cylinder(64, radius=25.0, seed=1).numpy()
    img, _ = oracle.normalize8(x)
    _check(rx, img)


def test_degenerate_images(rx):
    _check(rx, np.zeros((20, 40), np.uint8))
    _check(rx, np.full((20, 40), 77, np.uint8))
    img = np.zeros((16, 64), np.uint8)
    img[:, 10:20] = 255   # an object touching the border on two sides
    _check(rx, img)
