"""roix_extract_roi_static: the ROI mask without any device allocation.

Callers that cannot allocate device memory when they need a mask (code
recording a CUDA graph in global capture mode, acquisition loops that must not
block on cudaMalloc's implicit synchronisation, processes whose device memory
belongs to another allocator) use this entry point. It keeps its scratch in a
32 MiB array inside the library. These tests call it through the C ABI and
compare it with roix_extract_roi, which allocates a workspace: the masks and
their voxel counts must be identical (integer output: bit-exact), on two calls
in a row that reuse the same shared scratch. This file is collected last.
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
