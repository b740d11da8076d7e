"""roix_extract_roi_static: the ROI mask without any device allocation.

Callers that cannot allocate device memory when they need a mask (acquisition
loops that must not block on cudaMalloc's implicit synchronisation, processes
whose device memory belongs to another allocator or a fixed budget) use this
entry point. It keeps its scratch in a 32 MiB array inside the library. These
tests call it through the C ABI and compare it with roix_extract_roi, which
allocates a workspace, and with the oracle: the masks and their voxel counts
must be identical (integer output: bit-exact), on two calls in a row that
reuse the same shared scratch, and at exactly the largest accepted size.
This file is collected last.
"""
from __future__ import annotations

import ctypes as C

import pytest
import torch

import phantom


def _static(L, x, cfg, mask, pop, stream=None):
    import paper_2602_15917_gb300 as roix
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    return L.roix_extract_roi_static(x.data_ptr() if x is not None else None,
                                     roix._dtype_code(x) if x is not None else 1,
                                     roix.dims_of(x.shape), C.byref(roix.roi_of(**cfg)),
                                     mask.data_ptr() if mask is not None else None,
                                     pop.data_ptr() if pop is not None else None, s)


def test_static_rejects_sizes_beyond_its_scratch():
    # argument checks come before any CUDA call: runs with or without a GPU
    import paper_2602_15917_gb300 as roix
    L = roix.lib()
    big = roix.Dims(4096, 4096, 17)  # 17 * 4096 rows of 128 words > 2^23 words
    rc = L.roix_extract_roi_static(None, 1, big, C.byref(roix.roi_of()), None, None, None)
    assert rc == 1  # ROIX_EINVAL, nothing enqueued
    # one word over the limit: 2^23 + 1 rows of one word each
    over = roix.Dims(32, (1 << 23) + 1, 1)
    rc = L.roix_extract_roi_static(None, 1, over, C.byref(roix.roi_of()), None, None, None)
    assert rc == 1


@pytest.mark.gpu
def test_static_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2602_15917_gb300 as roix
    L = roix.lib()
    r = roix.Roix(0)
    cases = [
        (phantom.ellipsoids(shape=(37, 45, 70), seed=5).cuda(),
         dict(threshold=0.1, dilate=1)),
        (phantom.projection(300, 2, seed=4).cuda(),
         dict(cmp="lt", threshold=57000, dark=100, dilate=0)),
    ]
    for x, cfg in cases:  # two calls in a row on the shared scratch
        ref_mask, ref_pop = r.extract_roi(x, **cfg)
        r.sync()
        words = ref_mask.numel()
        mask = torch.full((words,), -1, dtype=torch.int32, device="cuda")
        pop = torch.full((1,), 7, dtype=torch.uint64, device="cuda")
        assert _static(L, x, cfg, mask, pop) == 0
        torch.cuda.synchronize()
        assert torch.equal(mask, ref_mask)
        assert int(pop.item()) == int(ref_pop.item())
    r.close()


@pytest.mark.gpu
def test_static_at_its_largest_size_equals_oracle():
    """Exactly 2^23 mask words (sixteen 4096 x 4096 uint8 images, 128 words a
    row): accepted, and the dilated mask equals the oracle's and
    roix_extract_roi's bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import numpy as np

    import oracle
    import paper_2602_15917_gb300 as roix
    L = roix.lib()
    rng = np.random.default_rng(11)
    xh = rng.integers(0, 256, (16, 4096, 4096), dtype=np.uint8)
    cfg = dict(threshold=250, dilate=1)
    x = torch.from_numpy(xh).cuda()
    words = int(L.roix_mask_words(roix.dims_of(x.shape)))
    assert words == 1 << 23
    mask = torch.full((words,), -1, dtype=torch.int32, device="cuda")
    pop = torch.full((1,), 7, dtype=torch.uint64, device="cuda")
    assert _static(L, x, cfg, mask, pop) == 0
    torch.cuda.synchronize()
    D = oracle.mask(xh, **cfg)
    want = np.packbits(D.reshape(16 * 4096, 4096), axis=1, bitorder="little").view(np.int32)
    assert np.array_equal(mask.cpu().numpy(), want.reshape(-1))
    assert int(pop.item()) == int(D.sum())
    r = roix.Roix(0)
    ref_mask, ref_pop = r.extract_roi(x, **cfg)
    r.sync()
    assert torch.equal(mask, ref_mask) and int(ref_pop.item()) == int(pop.item())
    r.close()
