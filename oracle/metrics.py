"""Evaluation metrics of the paper, on the CPU (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module. Plain numpy (and scipy's exact Euclidean
distance transform as a library step), float64 throughout.

* ``confusion`` / ``roi_metrics``: the ROI quality metrics of Sec. 5.2 (DSC,
  IoU, sensitivity, specificity, accuracy, Cohen's kappa with the chance term
  f_c, AUC from one operating point, average Hausdorff distance) between a
  predicted mask A and a ground-truth mask B, exactly as the section's
  equations write them.
* ``ssim``: the structural similarity of Sec. 5.6, in the form of Wang, Bovik,
  Sheikh and Simoncelli (2004): Gaussian window 11 x 11, sigma 1.5, K1 = 0.01,
  K2 = 0.03, population statistics, averaged over the positions where the
  window lies inside the image, per 2D slice (z), all slices weighted alike.

Where a ratio has a zero denominator (an empty set) the metric is NaN; the
distance terms of an empty set are NaN too.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

SSIM_RADIUS = 5
SSIM_SIGMA = 1.5
SSIM_K1, SSIM_K2 = 0.01, 0.03


def _div(a: float, b: float) -> float:
    with np.errstate(divide="ignore", invalid="ignore"):
        return float(np.float64(a) / np.float64(b))


def confusion(A: np.ndarray, B: np.ndarray):
    """TP, FP, FN, TN of prediction A against ground truth B (Sec. 5.2)."""
    A = np.asarray(A).astype(bool)
    B = np.asarray(B).astype(bool)
    tp = int(np.count_nonzero(A & B))
    fp = int(np.count_nonzero(A & ~B))
    fn = int(np.count_nonzero(~A & B))
    tn = int(A.size - tp - fp - fn)
    return tp, fp, fn, tn


def distance_sums(A: np.ndarray, B: np.ndarray):
    """(sum over a in A of min_b d(a, b), sum over b in B of min_a d(b, a)),
    d Euclidean on the voxel grid; NaN for an empty set on either side."""
    A = np.asarray(A).astype(bool)
    B = np.asarray(B).astype(bool)
    if not A.any() or not B.any():
        return float("nan"), float("nan")
    dB = ndimage.distance_transform_edt(~B)  # distance to the nearest voxel of B
    dA = ndimage.distance_transform_edt(~A)
    return float(np.sum(dB[A], dtype=np.float64)), float(np.sum(dA[B], dtype=np.float64))


def roi_metrics(A: np.ndarray, B: np.ndarray) -> dict:
    """The Sec. 5.2 equations, in their printed order of operations."""
    tp, fp, fn, tn = confusion(A, B)
    TP, FP, FN, TN = (np.float64(v) for v in (tp, fp, fn, tn))
    total = TP + TN + FN + FP
    fc = _div((TN + FN) * (TN + FP) + (FP + TP) * (FN + TP), total)
    sAB, sBA = distance_sums(A, B)
    nA, nB = tp + fp, tp + fn
    ahd = max(_div(sAB, nA), _div(sBA, nB)) if nA and nB else float("nan")
    return {
        "tp": tp, "fp": fp, "fn": fn, "tn": tn,
        "dsc": _div(2.0 * TP, (TP + FP) + (TP + FN)),
        "iou": _div(TP, TP + FP + FN),
        "sensitivity": _div(TP, TP + FN),
        "specificity": _div(TN, TN + FP),
        "accuracy": _div(TP + TN, TP + TN + FP + FN),
        "kappa": _div((TP + TN) - fc, (TP + TN + FN + FP) - fc),
        "auc": 1.0 - 0.5 * (_div(FP, FP + TN) + _div(FN, FN + TP)),
        "ahd": ahd,
        "sum_ab": sAB, "sum_ba": sBA,
    }


def gaussian_window() -> np.ndarray:
    """1D Gaussian taps, radius 5, sigma 1.5, normalised to sum 1."""
    t = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * SSIM_SIGMA * SSIM_SIGMA))
    return g / g.sum()


def ssim_map(x: np.ndarray, y: np.ndarray, data_range: float) -> np.ndarray:
    """SSIM at every position of one 2D slice where the window fits."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    g = gaussian_window()

    def filt(v):
        v = ndimage.correlate1d(v, g, axis=0, mode="constant")
        return ndimage.correlate1d(v, g, axis=1, mode="constant")

    r = SSIM_RADIUS
    sl = (slice(r, x.shape[0] - r), slice(r, x.shape[1] - r))
    mx, my = filt(x)[sl], filt(y)[sl]
    sxx = filt(x * x)[sl] - mx * mx
    syy = filt(y * y)[sl] - my * my
    sxy = filt(x * y)[sl] - mx * my
    c1 = (SSIM_K1 * data_range) ** 2
    c2 = (SSIM_K2 * data_range) ** 2
    return ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))


def ssim(x: np.ndarray, y: np.ndarray, data_range: float) -> float:
    """Mean SSIM over every valid window position of every 2D slice."""
    x = np.asarray(x)
    y = np.asarray(y)
    if x.ndim == 2:
        x, y = x[None], y[None]
    if x.shape[1] < 2 * SSIM_RADIUS + 1 or x.shape[2] < 2 * SSIM_RADIUS + 1:
        return float("nan")
    tot, cnt = 0.0, 0
    for z in range(x.shape[0]):
        m = ssim_map(x[z], y[z], data_range)
        tot += float(m.sum(dtype=np.float64))
        cnt += m.size
    return tot / cnt
