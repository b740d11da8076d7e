"""The C-ABI library loads and exports every entry point include/roix.h
declares; host-side helpers (no GPU calls)."""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "roix.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(roix_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_15917_gb300 import _build
    return _build.build()


def test_every_declared_symbol_is_exported(libpath):
    declared = _declared()
    assert "roix_compress" in declared and "roix_decode" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(roix_\w+)", out))
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    L = C.CDLL(libpath)
    for s in declared:
        assert getattr(L, s) is not None


def test_binding_knows_every_declared_symbol(libpath):
    import paper_2602_15917_gb300 as roix
    assert sorted(roix.symbols()) == _declared()
    L = roix.lib()
    for s in roix.symbols():
        assert getattr(L, s) is not None


def test_host_helpers_without_gpu(libpath):
    import paper_2602_15917_gb300 as roix
    L = roix.lib()
    d = roix.dims_of((3, 5, 70))
    assert L.roix_mask_words(d) == 15 * 3
    p = roix.params_of()
    b = L.roix_compress_bound(1, d, C.byref(p))
    assert b > 256 + 1024 + 3 * 5 * 70 * 12
    assert L.roix_status_string(3) == b"output buffer too small"
    ws = L.roix_workspace_size(1, d, C.byref(roix.roi_of()), C.byref(p), int(b))
    assert ws > 3 * 5 * 70 * 6
    # invalid parameters are refused before anything is enqueued
    assert L.roix_workspace_size(1, roix.Dims(70000, 1, 1), C.byref(roix.roi_of()),
                                 C.byref(p), 0) == 0
    bad = roix.params_of(chunk=1000)
    assert L.roix_workspace_size(1, d, C.byref(roix.roi_of()), C.byref(bad), 0) == 0


def test_ctx_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2602_15917_gb300 as roix
    h = C.c_void_p()
    assert roix.lib().roix_ctx_create(0, C.byref(h)) == 6  # ROIX_ECUDA
    with pytest.raises(roix.RoixError):
        roix.Roix(0)


def test_server_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2602_15917_gb300 as roix
    with pytest.raises(roix.RoixError):
        roix.RoixServer(0, hbm_budget=1 << 30, lanes=2)
    h = C.c_void_p()
    bad = roix.ServerConfig(1 << 30, 0, 8)  # no lanes
    assert roix.lib().roix_server_create(0, C.byref(bad), C.byref(h)) == 1


def test_slab_workspace_size_checks_arguments(libpath):
    import paper_2602_15917_gb300 as roix
    L = roix.lib()
    d = roix.dims_of((70, 30, 40))
    p = roix.params_of()
    ok = L.roix_slabs_workspace_size(1, d, 16, C.byref(roix.roi_of()), C.byref(p), 1 << 20)
    # at least the pixel sections and symbols of every slab and the whole mask
    assert ok >= 70 * 30 * 40 * 6 + 70 * 30 * 2 * 4
    assert L.roix_slabs_workspace_size(1, d, 0, C.byref(roix.roi_of()), C.byref(p), 0) == 0
    assert L.roix_slabs_workspace_size(1, d, 16, C.byref(roix.roi_of(keep="largest")),
                                       C.byref(p), 0) == 0
    assert L.roix_slabs_workspace_size(3, d, 16, C.byref(roix.roi_of()), C.byref(p), 0) == 0
