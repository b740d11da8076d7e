"""Pins of the CPU evaluation metrics (oracle/metrics.py) against things other
than themselves: textbook tables, identities between the Sec. 5.2 metrics,
brute-force distances, a closed form of the average Hausdorff distance, and a
direct window-by-window SSIM (Wang et al. 2004)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import metrics as M

def _masks_with_counts(tp, fp, fn, tn):
    A = np.array([1] * tp + [1] * fp + [0] * fn + [0] * tn, np.uint8)
    B = np.array([1] * tp + [0] * fp + [1] * fn + [0] * tn, np.uint8)
    return A, B

def test_confusion_counts():
    A, B = _masks_with_counts(7, 3, 2, 11)
    assert M.confusion(A, B) == (7, 3, 2, 11)

def test_kappa_textbook_table():
    # the classic 2x2 agreement table 20 / 5 / 10 / 15 has Cohen's kappa 0.4
    A, B = _masks_with_counts(20, 10, 5, 15)
    m = M.roi_metrics(A.reshape(1, -1), B.reshape(1, -1))
    assert m["kappa"] == pytest.approx(0.4, abs=1e-15)
    assert m["accuracy"] == pytest.approx(0.7, abs=1e-15)

@pytest.mark.parametrize("seed", range(6))
def test_identities_between_metrics(seed):
    rng = np.random.default_rng(seed)
    A = (rng.random((9, 13, 17)) < 0.3).astype(np.uint8)
    B = (rng.random((9, 13, 17)) < 0.35).astype(np.uint8)
    m = M.roi_metrics(A, B)
    assert m["iou"] == pytest.approx(m["dsc"] / (2 - m["dsc"]), rel=1e-12)
    assert m["auc"] == pytest.approx((m["sensitivity"] + m["specificity"]) / 2, rel=1e-12)
    # kappa from observed and expected agreement written the textbook way
    n = A.size
    po = (m["tp"] + m["tn"]) / n
    pa, pb = (m["tp"] + m["fp"]) / n, (m["tp"] + m["fn"]) / n
    pe = pa * pb + (1 - pa) * (1 - pb)
    assert m["kappa"] == pytest.approx((po - pe) / (1 - pe), rel=1e-12)

def _brute_sums(A, B):
    pa = np.argwhere(A)
    pb = np.argwhere(B)
    d = np.sqrt(((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1))
    return d.min(1).sum(), d.min(0).sum()

@pytest.mark.parametrize("shape,seed", [((20, 23), 0), ((5, 9, 11), 1), ((1, 30, 7), 2),
                                        ((6, 6, 6), 3)])
def test_distance_sums_brute_force(shape, seed):
    rng = np.random.default_rng(seed)
    A = rng.random(shape) < 0.2
    B = rng.random(shape) < 0.1
    A.flat[0] = True
    B.flat[-1] = True
    s1, s2 = M.distance_sums(A, B)
    b1, b2 = _brute_sums(A, B)
    assert s1 == pytest.approx(b1, rel=1e-12) and s2 == pytest.approx(b2, rel=1e-12)

@pytest.mark.parametrize("m,k,dim", [(10, 1, 2), (10, 3, 2), (8, 5, 3), (12, 2, 3)])
def test_ahd_shifted_square_closed_form(m, k, dim):
    shape = (m + k + 4,) * dim
    A = np.zeros(shape, bool)
    B = np.zeros(shape, bool)
    sl = tuple(slice(2, 2 + m) for _ in range(dim))
    A[sl] = True
    sh = list(sl)
    sh[-1] = slice(2 + k, 2 + m + k)
    B[tuple(sh)] = True
    assert M.roi_metrics(A, B)["ahd"] == pytest.approx(k * (k + 1) / (2 * m), rel=1e-12)

def test_empty_sets_are_nan():
    A = np.zeros((4, 4), np.uint8)
    B = np.zeros((4, 4), np.uint8)
    B[1, 1] = 1
    m = M.roi_metrics(A, B)
    assert np.isnan(m["ahd"]) and m["dsc"] == 0.0 and np.isnan(m["sum_ab"])
    m = M.roi_metrics(A, A)
    assert np.isnan(m["dsc"]) and m["specificity"] == 1.0

def _ssim_direct(x, y, L):
    """Every window position, every tap: weighted sums written out."""
    g = M.gaussian_window()
    w = np.outer(g, g)
    r = M.SSIM_RADIUS
    c1, c2 = (M.SSIM_K1 * L) ** 2, (M.SSIM_K2 * L) ** 2
    vals = []
    for i in range(r, x.shape[0] - r):
        for j in range(r, x.shape[1] - r):
            a = x[i - r:i + r + 1, j - r:j + r + 1].astype(np.float64)
            b = y[i - r:i + r + 1, j - r:j + r + 1].astype(np.float64)
            mx, my = (w * a).sum(), (w * b).sum()
            vx = (w * (a - mx) ** 2).sum()
            vy = (w * (b - my) ** 2).sum()
            cxy = (w * (a - mx) * (b - my)).sum()
            vals.append(((2 * mx * my + c1) * (2 * cxy + c2)) /
                        ((mx * mx + my * my + c1) * (vx + vy + c2)))
    return float(np.mean(vals))

@pytest.mark.parametrize("seed", range(3))
def test_ssim_equals_direct_windows(seed):
    rng = np.random.default_rng(seed)
    x = rng.random((19, 24)) * 200
    y = x + rng.normal(0, 10, x.shape)
    assert M.ssim(x, y, 255.0) == pytest.approx(_ssim_direct(x, y, 255.0), abs=1e-12)
    assert M.ssim(y, x, 255.0) == pytest.approx(M.ssim(x, y, 255.0), abs=1e-15)

def test_ssim_identity_and_constants():
    rng = np.random.default_rng(9)
    x = rng.random((3, 16, 20)).astype(np.float32)
    assert M.ssim(x, x, 1.0) == pytest.approx(1.0, abs=1e-12)
    a, b, L = 100.0, 110.0, 255.0
    c1 = (M.SSIM_K1 * L) ** 2
    want = (2 * a * b + c1) / (a * a + b * b + c1)
    assert M.ssim(np.full((12, 12), a), np.full((12, 12), b), L) == pytest.approx(want, rel=1e-12)
    assert np.isnan(M.ssim(np.zeros((10, 30)), np.zeros((10, 30)), 1.0))

def test_gaussian_window():
    g = M.gaussian_window()
    assert g.size == 11 and abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert g[5] / g[4] == pytest.approx(np.exp(1 / (2 * 1.5 ** 2)), rel=1e-14)
