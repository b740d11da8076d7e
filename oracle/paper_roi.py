"""Paper-mode region of interest on the CPU (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module. Plain numpy, with ``scipy.ndimage.label``
as the connected-component step. Every 2D slice (z) of an 8-bit image is an
image of its own:

1. multi-Otsu thresholds (Sec. 4.1.3, after Liao, Chen and Chung 2001): three
   classes C0 = [0, t1], C1 = (t1, t2], C2 = (t2, 255] of the 256-bin
   histogram, chosen to maximise the between-class variance, i.e. the sum over
   the classes of (sum of values)^2 / (count); empty classes add 0; among
   equal maxima the smallest (t1, t2) in lexicographic order;
2. binarisation M = [I_n > t1] (Sec. 4.1.4: the object is above the cut-off);
3. the object's outer boundary (Sec. 4.2.1, external contours only): holes
   of M are filled, a hole being background (4-connected) that does not
   reach the slice border;
4. the largest object: the 8-connected component of the filled mask with the
   most pixels (its area inside the external contour), ties to the one
   holding the smallest raster index;
5. one span per row (Sec. 4.2.2, G(i) = [i, x_start, x_end]): every row
   keeps [x_start, x_end) from the object's leftmost to its rightmost pixel,
   gaps included.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

_FOUR = ndimage.generate_binary_structure(2, 1)
_EIGHT = ndimage.generate_binary_structure(2, 2)


def multiotsu(hist: np.ndarray):
    """Thresholds (t1, t2) of a 256-bin histogram (step 1)."""
    h = np.asarray(hist, np.int64)
    v = np.arange(256, dtype=np.int64)
    P = np.cumsum(h)
    S = np.cumsum(h * v)
    best, arg = -1.0, (0, 1)
    for t1 in range(0, 254):
        for t2 in range(t1 + 1, 255):
            counts = (P[t1], P[t2] - P[t1], P[255] - P[t2])
            sums = (S[t1], S[t2] - S[t1], S[255] - S[t2])
            f = 0.0
            for c, s in zip(counts, sums):
                term = np.float64(s) * np.float64(s) / np.float64(c) if c else np.float64(0.0)
                f = np.float64(f) + term
            if f > best:
                best, arg = f, (t1, t2)
    return arg


def fill_holes(M: np.ndarray) -> np.ndarray:
    """Step 3 on one slice: background 4-components off the border become object."""
    bg, n = ndimage.label(~M.astype(bool), structure=_FOUR)
    border = set(np.unique(np.concatenate([bg[0], bg[-1], bg[:, 0], bg[:, -1]]))) - {0}
    keep_bg = np.isin(bg, sorted(border))
    return ~keep_bg


def largest(F: np.ndarray) -> np.ndarray:
    """Step 4 on one slice."""
    lab, n = ndimage.label(F.astype(bool), structure=_EIGHT)
    if n == 0:
        return np.zeros(F.shape, bool)
    sizes = np.bincount(lab.ravel())[1:]
    first = np.full(n, np.iinfo(np.int64).max)
    idx = np.flatnonzero(lab.ravel())
    np.minimum.at(first, lab.ravel()[idx] - 1, idx)
    best = max(range(n), key=lambda k: (sizes[k], -first[k]))
    return lab == best + 1


def spans(K: np.ndarray) -> np.ndarray:
    """Step 5 on one slice."""
    D = np.zeros(K.shape, bool)
    for y in range(K.shape[0]):
        xs = np.flatnonzero(K[y])
        if xs.size:
            D[y, xs[0]:xs[-1] + 1] = True
    return D


def paper_mask(img: np.ndarray):
    """Steps 1-5 on every slice of a uint8 image (2D or 3D, z first); returns
    (mask as uint8, thresholds as an int array of shape (nz, 2))."""
    img = np.asarray(img)
    if img.dtype != np.uint8:
        raise TypeError("uint8 image")
    vol = img[None] if img.ndim == 2 else img
    out = np.zeros(vol.shape, np.uint8)
    thr = np.zeros((vol.shape[0], 2), np.int64)
    for z in range(vol.shape[0]):
        sl = vol[z]
        t1, t2 = multiotsu(np.bincount(sl.ravel(), minlength=256))
        thr[z] = (t1, t2)
        out[z] = spans(largest(fill_holes(sl > t1)))
    return (out[0] if img.ndim == 2 else out), thr
