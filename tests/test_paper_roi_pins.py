"""Pins of the paper-mode ROI oracle (oracle/paper_roi.py): multi-Otsu against
the textbook between-class variance written with class probabilities and
means, a three-spike histogram with a closed-form answer, hole filling against
scipy's binary_fill_holes, and hand-made largest-object and span cases."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import ndimage

from oracle import paper_roi as PR


def _otsu_textbook(h):
    p = h / h.sum()
    v = np.arange(256)
    mu_t = (p * v).sum()
    best, arg = -1.0, None
    for t1 in range(254):
        for t2 in range(t1 + 1, 255):
            s = 0.0
            for lo, hi in ((0, t1 + 1), (t1 + 1, t2 + 1), (t2 + 1, 256)):
                w = p[lo:hi].sum()
                if w > 0:
                    mu = (p[lo:hi] * v[lo:hi]).sum() / w
                    s += w * (mu - mu_t) ** 2
            if s > best + 1e-12:
                best, arg = s, (t1, t2)
    return arg


@pytest.mark.parametrize("seed", range(3))
def test_multiotsu_equals_textbook_variance(seed):
    rng = np.random.default_rng(seed)
    vals = np.concatenate([rng.normal(40, 8, 4000), rng.normal(120, 10, 3000),
                           rng.normal(200, 6, 2000)])
    h = np.bincount(np.clip(np.rint(vals), 0, 255).astype(int), minlength=256)
    t = PR.multiotsu(h)
    assert t == _otsu_textbook(h.astype(np.float64))
    assert 40 < t[0] < 120 < t[1] < 200


def test_multiotsu_three_spikes_closed_form():
    h = np.zeros(256, np.int64)
    h[10], h[100], h[200] = 5, 3, 7
    # every t1 in [10, 99], t2 in [100, 199] separates the spikes perfectly;
    # the smallest such pair is chosen
    assert PR.multiotsu(h) == (10, 100)


@pytest.mark.parametrize("seed", range(4))
def test_fill_holes_equals_scipy(seed):
    rng = np.random.default_rng(seed)
    M = ndimage.binary_dilation(rng.random((40, 50)) < 0.08, iterations=2)
    assert np.array_equal(PR.fill_holes(M), ndimage.binary_fill_holes(M))


def test_largest_counts_filled_area():
    F = np.zeros((30, 60), bool)
    F[2:22, 2:22] = True     # a ring: 20 x 20 outline, 2 thick (144 pixels) ...
    F[4:20, 4:20] = False
    F[5:25, 30:40] = True    # ... and a solid 20 x 10 block (200 pixels)
    K = PR.largest(PR.fill_holes(F))
    assert K[10, 10] and not K[10, 35]  # filled ring: 400 pixels beat 200


def test_largest_tie_smallest_index_and_diagonal():
    F = np.zeros((10, 10), bool)
    F[1, 1] = F[2, 2] = True   # diagonal neighbours: one component (8-connected)
    F[6, 6] = F[6, 7] = True   # same size, later
    K = PR.largest(F)
    assert K[1, 1] and K[2, 2] and not K[6, 6]


def test_spans_keep_gaps():
    K = np.zeros((3, 12), bool)
    K[0, [2, 3, 9]] = True
    K[2, 5] = True
    D = PR.spans(K)
    assert D[0].tolist() == [False, False] + [True] * 8 + [False, False]
    assert not D[1].any() and D[2].tolist() == [i == 5 for i in range(12)]


def test_paper_mask_disk_with_hole():
    yy, xx = np.mgrid[:64, :64]
    r = np.hypot(yy - 32, xx - 32)
    img = np.where(r < 20, 200, 20).astype(np.uint8)
    img[r < 6] = 20                    # a hole in the object
    img[5, 5] = 200                    # an isolated speck
    img[(yy > 55) & (xx > 55)] = 110   # a third grey level
    D, thr = PR.paper_mask(img)
    want = PR.spans(r < 20)
    assert np.array_equal(D.astype(bool), want)
    assert thr.shape == (1, 2)
