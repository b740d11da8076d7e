"""Python binding of libroix, the GB300 (sm_103a) ROIX-Comp hot path.

The binding only marshals arguments: every step runs in the CUDA kernels of
``csrc/`` behind the C ABI of ``include/roix.h``. PyTorch supplies device
memory and streams. There is no CPU fallback: if ``libroix.so`` has not been
built (``__graft_entry__.build()``) or no GPU is present, the calls raise.

Two layers:
* ``lib()`` - the ctypes handle; its functions carry the C names
  (``roix_compress``, ``roix_extract_roi``, ``roix_compact``,
  ``roix_quantize``, ``roix_encode``, ``roix_decode`` ...) and take raw pointers.
* ``Roix`` - the same calls on torch tensors, with the ROI / error-bound /
  coder settings given as keyword arguments (``eb``, ``eb_mode``, ``cmp``,
  ``threshold``, ``keep``, ``connectivity``, ``dilate``, ``dark``, ``fill``,
  ``radius``, ``chunk``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import _build

F32, U16, U8 = 1, 2, 3
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory",
          3: "output buffer too small", 4: "corrupt container", 5: "wait timed out",
          6: "CUDA error", 7: "busy"}


class RoixError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}{': ' + msg if msg else ''}")
        self.status = status


class Dims(C.Structure):
    _fields_ = [("nx", C.c_uint64), ("ny", C.c_uint64), ("nz", C.c_uint64)]


class Roi(C.Structure):
    _fields_ = [("cmp", C.c_int32), ("keep", C.c_int32), ("connectivity", C.c_int32),
                ("dilate", C.c_int32), ("threshold", C.c_double), ("dark", C.c_double)]


class Eb(C.Structure):
    _fields_ = [("mode", C.c_int32), ("value", C.c_double)]


class Params(C.Structure):
    _fields_ = [("radius", C.c_uint32), ("chunk", C.c_uint32), ("fill", C.c_double),
                ("predictor", C.c_uint32)]


class Item(C.Structure):
    _fields_ = [("in_", C.c_void_p), ("dims", Dims), ("out", C.c_void_p), ("cap", C.c_uint64),
                ("size_dev", C.c_void_p)]


class RoiMetrics(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("tp", "fp", "fn", "tn")] + \
        [(k, C.c_double) for k in ("dsc", "iou", "sensitivity", "specificity", "accuracy",
                                   "kappa", "auc", "ahd", "sum_ab", "sum_ba")]


class GreedyItem(C.Structure):
    _fields_ = [("pixels", C.c_void_p), ("mask", C.c_void_p), ("dims", Dims),
                ("q_out", C.c_void_p), ("n_dev", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("lanes", C.c_uint32), ("max_batch", C.c_uint32)]


class Request(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("in_", C.c_void_p), ("dtype", C.c_int32), ("dims", Dims),
                ("roi", Roi), ("eb", Eb), ("params", Params), ("out", C.c_void_p),
                ("cap", C.c_uint64)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("size", C.c_uint64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("bytes_in", C.c_uint64), ("max_queue", C.c_uint64), ("pending", C.c_uint64),
                ("budget_bytes", C.c_uint64), ("in_use_bytes", C.c_uint64)]


class Tuning(C.Structure):
    _fields_ = [(k, C.c_uint32) for k in ("front_words", "thr_blocks_per_sm",
                                          "flat_blocks_per_sm", "sym_blocks_per_sm",
                                          "pack_blocks_per_sm", "front_kernel")]


class EbInfo(C.Structure):
    _fields_ = [("eb_abs", C.c_double), ("vmin", C.c_double), ("vmax", C.c_double),
                ("two_eb", C.c_float), ("inv2eb", C.c_float), ("bound", C.c_float),
                ("eb_int", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libroix (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libroix.so is not built: call __graft_entry__.build()")
            L = C.CDLL(_build.LIB)
            P, u64, i32, st = C.c_void_p, C.c_uint64, C.c_int32, C.c_int
            D, R, E, PR = Dims, C.POINTER(Roi), C.POINTER(Eb), C.POINTER(Params)
            sig = {
                "roix_ctx_create": (st, [i32, C.POINTER(P)]),
                "roix_ctx_destroy": (st, [P]),
                "roix_reserve": (st, [P, C.c_size_t]),
                "roix_workspace_size": (C.c_size_t, [i32, D, R, PR, u64]),
                "roix_sync": (st, [P, P]),
                "roix_set_wait_limit": (st, [P, C.c_uint32]),
                "roix_debug_hold_scans": (st, [P, C.c_int]),
                "roix_last_error": (C.c_char_p, [P]),
                "roix_status_string": (C.c_char_p, [st]),
                "roix_mask_words": (u64, [D]),
                "roix_compress_bound": (u64, [i32, D, PR]),
                "roix_extract_roi": (st, [P, P, i32, D, R, P, P, P]),
                "roix_compact": (st, [P, P, i32, D, P, P, P, P, u64, P, P]),
                "roix_quantize": (st, [P, P, i32, u64, P, E, C.c_double, P, P, P, P]),
                "roix_encode": (st, [P, P, P, P, u64, P, P, P, P, i32, D, R, E, PR, P, u64, P,
                                     P]),
                "roix_decode": (st, [P, P, u64, P, i32, D, P]),
                "roix_compress": (st, [P, P, i32, D, R, E, PR, P, u64, P, P]),
                "roix_profile": (st, [P, C.c_int]),
                "roix_profile_read": (C.c_int, [P, C.POINTER(C.c_float), C.c_int]),
                "roix_extract_roi_static": (st, [P, i32, D, R, P, P, P]),
                "roix_compress_batch": (st, [P, C.c_uint32, C.POINTER(Item), i32, R, E, PR, P]),
                "roix_server_create": (st, [i32, C.POINTER(ServerConfig), C.POINTER(P)]),
                "roix_server_submit": (st, [P, C.POINTER(Request)]),
                "roix_server_poll": (C.c_uint32, [P, C.POINTER(Completion), C.c_uint32]),
                "roix_server_drain": (st, [P, C.c_double]),
                "roix_server_get_stats": (st, [P, C.POINTER(ServerStats)]),
                "roix_server_destroy": (st, [P]),
                "roix_normalize8": (st, [P, P, i32, D, C.c_double, P, P, P]),
                "roix_greedy_quantize": (st, [P, P, P, D, C.c_double, P, P, P]),
                "roix_greedy_quantize_batch": (st, [P, C.c_uint32, C.POINTER(GreedyItem),
                                                    C.c_double, P]),
                "roix_roi_quality": (st, [P, P, P, D, C.c_int, P, P]),
                "roix_extract_roi_paper": (st, [P, P, D, P, P, P, P]),
                "roix_ssim": (st, [P, P, P, i32, D, C.c_double, P, P]),
                "roix_compress_slabs": (st, [P, P, i32, D, u64, R, E, PR, C.POINTER(P),
                                             C.POINTER(u64), P, P]),
                "roix_slabs_workspace_size": (C.c_size_t, [i32, D, u64, R, PR, u64]),
                "roix_get_tuning": (st, [P, C.POINTER(Tuning)]),
                "roix_set_tuning": (st, [P, C.POINTER(Tuning)]),
                "roix_tune": (st, [P, C.c_uint32, C.POINTER(Item), i32, R, E, PR, C.c_uint32,
                                   C.c_char_p, C.POINTER(Tuning), P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def symbols():
    """Names of the entry points the binding knows (all declared in roix.h)."""
    return ["roix_ctx_create", "roix_ctx_destroy", "roix_reserve", "roix_workspace_size",
            "roix_sync", "roix_set_wait_limit", "roix_debug_hold_scans", "roix_last_error", "roix_status_string", "roix_mask_words",
            "roix_compress_bound", "roix_extract_roi", "roix_compact", "roix_quantize",
            "roix_encode", "roix_decode", "roix_compress", "roix_profile",
            "roix_profile_read", "roix_extract_roi_static", "roix_compress_batch",
            "roix_server_create", "roix_server_submit", "roix_server_poll", "roix_server_drain",
            "roix_server_get_stats", "roix_server_destroy", "roix_normalize8",
            "roix_greedy_quantize", "roix_greedy_quantize_batch", "roix_roi_quality",
            "roix_ssim", "roix_extract_roi_paper", "roix_compress_slabs",
            "roix_slabs_workspace_size", "roix_get_tuning", "roix_set_tuning", "roix_tune"]


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.uint16:
        return U16
    if t.dtype == torch.uint8:
        return U8
    raise TypeError("float32, uint16 or uint8 tensors only")


def dims_of(shape) -> Dims:
    shape = tuple(int(s) for s in shape)
    if len(shape) == 1:
        return Dims(shape[0], 1, 1)
    if len(shape) == 2:
        return Dims(shape[1], shape[0], 1)
    if len(shape) == 3:
        return Dims(shape[2], shape[1], shape[0])
    raise ValueError("1D, 2D or 3D volumes only")


def roi_of(cmp="gt", threshold=0.1, keep="all", connectivity=26, dilate=1, dark=0.0, **_) -> Roi:
    return Roi(0 if cmp == "gt" else 1, 0 if keep == "all" else 1, int(connectivity),
               int(dilate), float(threshold), float(dark))


def eb_of(eb=1e-3, eb_mode="abs", **_) -> Eb:
    return Eb(0 if eb_mode == "abs" else 1, float(eb))


def params_of(radius=512, chunk=4096, fill=0.0, predictor=1, **_) -> Params:
    return Params(int(radius), int(chunk), float(fill), int(predictor))


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Roix:
    """A libroix context on one GPU, with tensor-level calls."""

    def __init__(self, device: int = 0):
        self.L = lib()
        self.device = device
        h = C.c_void_p()
        self._check(self.L.roix_ctx_create(int(device), C.byref(h)), ctx=False)
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            self.L.roix_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status: int, ctx: bool = True):
        if status != 0:
            msg = self.L.roix_last_error(self.ctx).decode() if ctx and self.ctx else ""
            raise RoixError(status, msg)

    def sync(self, stream=None):
        self._check(self.L.roix_sync(self.ctx, _stream(stream)))

    def set_wait_limit(self, polls: int = 0):
        """roix_set_wait_limit: polls of a bounded device wait before it gives
        up with ROIX_ETIMEOUT (0: the library's default)."""
        self._check(self.L.roix_set_wait_limit(self.ctx, int(polls)))

    def debug_hold_scans(self, on: bool = True):
        """roix_debug_hold_scans: test hook that leaves the first tile of every
        tile scan unpublished, so that the bounded waits run out."""
        self._check(self.L.roix_debug_hold_scans(self.ctx, int(on)))

    def reserve(self, nbytes: int):
        self._check(self.L.roix_reserve(self.ctx, int(nbytes)))

    def profile(self, on: bool = True):
        self._check(self.L.roix_profile(self.ctx, int(on)))

    def profile_read(self, n: int = 16):
        buf = (C.c_float * n)()
        k = self.L.roix_profile_read(self.ctx, buf, n)
        return [buf[i] for i in range(k)]

    def bound(self, shape, dtype=torch.float32, **cfg) -> int:
        code = F32 if dtype == torch.float32 else U16
        return int(self.L.roix_compress_bound(code, dims_of(shape), C.byref(params_of(**cfg))))

    def workspace_size(self, shape, dtype=torch.float32, cap=None, **cfg) -> int:
        code = F32 if dtype == torch.float32 else U16
        cap = self.bound(shape, dtype, **cfg) if cap is None else cap
        return int(self.L.roix_workspace_size(code, dims_of(shape), C.byref(roi_of(**cfg)),
                                              C.byref(params_of(**cfg)), int(cap)))

    # ------------------------------------------------------------- autotuner
    def get_tuning(self) -> dict:
        t = Tuning()
        self._check(self.L.roix_get_tuning(self.ctx, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        """roix_set_tuning with the given fields changed: front_words (mask words
        per compaction tile), thr_blocks_per_sm / flat_blocks_per_sm
        (binarisation, row and flat forms), sym_blocks_per_sm,
        pack_blocks_per_sm (0: as many as fit), front_kernel (compaction
        counts: 0 a block per tile, 1 a warp per tile). None of them changes an
        output byte; values out of range raise RoixError (status 1)."""
        cur = self.get_tuning()
        cur.update(kw)
        self._check(self.L.roix_set_tuning(self.ctx, C.byref(Tuning(**cur))))

    def tune(self, xs, outs=None, caps=None, sizes=None, reps: int = 5, cache: str | None = None,
             stream=None, **cfg) -> dict:
        """roix_tune on the batch xs (as compress_batch); returns the tuning."""
        n = len(xs)
        dev = xs[0].device
        if outs is None:
            caps = [x.numel() * x.element_size() + 65536 for x in xs] if caps is None else caps
            outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
        caps = [o.numel() for o in outs] if caps is None else caps
        if sizes is None:
            sizes = torch.zeros(n, dtype=torch.uint64, device=dev)
        arr = (Item * n)()
        for i, x in enumerate(xs):
            arr[i] = Item(x.data_ptr(), dims_of(x.shape), outs[i].data_ptr(), int(caps[i]),
                          sizes.data_ptr() + 8 * i)
        t = Tuning()
        self._check(self.L.roix_tune(self.ctx, n, arr, _dtype_code(xs[0]), C.byref(roi_of(**cfg)),
                                     C.byref(eb_of(**cfg)), C.byref(params_of(**cfg)), int(reps),
                                     cache.encode() if cache else None, C.byref(t),
                                     _stream(stream)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    # ------------------------------------------------------------ fused path
    def compress(self, x: torch.Tensor, out: torch.Tensor | None = None, cap: int | None = None,
                 size: torch.Tensor | None = None, stream=None, **cfg):
        """Enqueues the whole compression of x; returns (out, size) with size a
        1-element uint64 device tensor holding the container's byte count."""
        assert x.is_cuda and x.is_contiguous()
        if out is None:
            cap = cap if cap is not None else x.numel() * x.element_size() + 65536
            out = torch.empty(cap, dtype=torch.uint8, device=x.device)
        cap = out.numel() if cap is None else cap
        if size is None:
            size = torch.zeros(1, dtype=torch.uint64, device=x.device)
        self._check(self.L.roix_compress(
            self.ctx, x.data_ptr(), _dtype_code(x), dims_of(x.shape), C.byref(roi_of(**cfg)),
            C.byref(eb_of(**cfg)), C.byref(params_of(**cfg)), out.data_ptr(), int(cap),
            size.data_ptr(), _stream(stream)))
        return out, size

    def compress_batch(self, xs, outs=None, caps=None, sizes: torch.Tensor | None = None,
                       stream=None, **cfg):
        """Enqueues the batched compression of the tensors xs (same dtype and
        settings); returns (outs, sizes) with sizes a uint64 device tensor."""
        n = len(xs)
        if n == 0:
            return [], torch.zeros(0, dtype=torch.uint64)
        dev = xs[0].device
        if outs is None:
            caps = [x.numel() * x.element_size() + 65536 for x in xs] if caps is None else caps
            outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in caps]
        caps = [o.numel() for o in outs] if caps is None else caps
        if sizes is None:
            sizes = torch.zeros(n, dtype=torch.uint64, device=dev)
        arr = (Item * n)()
        for i, x in enumerate(xs):
            assert x.is_cuda and x.is_contiguous() and x.dtype == xs[0].dtype
            arr[i] = Item(x.data_ptr(), dims_of(x.shape), outs[i].data_ptr(), int(caps[i]),
                          sizes.data_ptr() + 8 * i)
        self._check(self.L.roix_compress_batch(
            self.ctx, n, arr, _dtype_code(xs[0]), C.byref(roi_of(**cfg)), C.byref(eb_of(**cfg)),
            C.byref(params_of(**cfg)), _stream(stream)))
        return outs, sizes

    def slabs_workspace_size(self, shape, slab_z: int, dtype=torch.float32, cap=None,
                             **cfg) -> int:
        code = F32 if dtype == torch.float32 else U16
        d = dims_of(shape)
        if cap is None:
            cap = self.bound((min(int(slab_z), int(d.nz)), d.ny, d.nx), dtype, **cfg)
        return int(self.L.roix_slabs_workspace_size(code, d, int(slab_z), C.byref(roi_of(**cfg)),
                                                    C.byref(params_of(**cfg)), int(cap)))

    def compress_slabs(self, x: torch.Tensor, slab_z: int, outs=None, caps=None,
                       sizes: torch.Tensor | None = None, stream=None, **cfg):
        """Enqueues the compression of the 3D tensor x in z-slabs of slab_z
        slices (whole-volume mask and error bound, one container per slab);
        returns (outs, sizes) with sizes a uint64 device tensor, one per slab."""
        assert x.is_cuda and x.is_contiguous() and x.dim() == 3
        nz = int(x.shape[0])
        ns = (nz + int(slab_z) - 1) // int(slab_z) if nz and int(slab_z) > 0 else 0
        if outs is None:
            if caps is None:
                caps = []
                for k in range(ns):  # the worst case: every voxel retained, every value a record
                    dz = min(int(slab_z), nz - k * int(slab_z))
                    caps.append(self.bound((dz, x.shape[1], x.shape[2]), x.dtype, **cfg))
            outs = [torch.empty(c, dtype=torch.uint8, device=x.device) for c in caps]
        caps = [o.numel() for o in outs] if caps is None else caps
        if sizes is None:
            sizes = torch.zeros(max(ns, 1), dtype=torch.uint64, device=x.device)
        po = (C.c_void_p * max(ns, 1))(*[o.data_ptr() for o in outs])
        pc = (C.c_uint64 * max(ns, 1))(*[int(c) for c in caps])
        self._check(self.L.roix_compress_slabs(
            self.ctx, x.data_ptr(), _dtype_code(x), dims_of(x.shape), int(slab_z),
            C.byref(roi_of(**cfg)), C.byref(eb_of(**cfg)), C.byref(params_of(**cfg)), po, pc,
            sizes.data_ptr(), _stream(stream)))
        return outs, sizes[:ns]

    def compress_bytes(self, x: torch.Tensor, **cfg) -> torch.Tensor:
        """compress + sync; returns the container as a uint8 device tensor. An
        output too small for the container is grown once to the size needed."""
        out, size = self.compress(x, **cfg)
        try:
            self.sync()
        except RoixError as e:
            if e.status != 3:
                raise
            need = int(size.item())
            out, size = self.compress(x, cap=need, out=torch.empty(need, dtype=torch.uint8,
                                                                   device=x.device), **cfg)
            self.sync()
        return out[:int(size.item())]

    def decode(self, buf: torch.Tensor, shape, dtype=torch.float32, size: int | None = None,
               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        assert buf.is_cuda and buf.dtype == torch.uint8
        if out is None:
            out = torch.empty(shape, dtype=dtype, device=buf.device)
        size = buf.numel() if size is None else size
        self._check(self.L.roix_decode(self.ctx, buf.data_ptr(), int(size), out.data_ptr(),
                                       _dtype_code(out), dims_of(shape), _stream(stream)))
        return out

    # ---------------------------------------------------------------- stages
    def extract_roi(self, x: torch.Tensor, stream=None, **cfg):
        d = dims_of(x.shape)
        words = int(self.L.roix_mask_words(d))
        mask = torch.empty(max(words, 1), dtype=torch.int32, device=x.device)
        pop = torch.zeros(1, dtype=torch.uint64, device=x.device)
        self._check(self.L.roix_extract_roi(self.ctx, x.data_ptr(), _dtype_code(x), d,
                                            C.byref(roi_of(**cfg)), mask.data_ptr(),
                                            pop.data_ptr(), _stream(stream)))
        return mask[:words], pop

    def compact(self, x: torch.Tensor, mask: torch.Tensor, bounds_cap: int | None = None,
                stream=None):
        d = dims_of(x.shape)
        rows = d.ny * d.nz
        bounds_cap = rows * (d.nx + 1) if bounds_cap is None else bounds_cap
        pixels = torch.empty(max(x.numel(), 1), dtype=x.dtype, device=x.device)
        counts = torch.empty(max(rows, 1), dtype=torch.uint16, device=x.device)
        bounds = torch.empty(max(bounds_cap, 1), dtype=torch.uint16, device=x.device)
        sizes = torch.zeros(2, dtype=torch.uint64, device=x.device)
        self._check(self.L.roix_compact(self.ctx, x.data_ptr(), _dtype_code(x), d,
                                        mask.data_ptr(), pixels.data_ptr(), counts.data_ptr(),
                                        bounds.data_ptr(), int(bounds_cap), sizes.data_ptr(),
                                        _stream(stream)))
        return pixels, counts[:rows], bounds, sizes

    def normalize8(self, x: torch.Tensor, dark: float = 0.0, out: torch.Tensor | None = None,
                   stream=None):
        """Sec. 4.1.2: the 8-bit image (uint8, shape of x) and I_max (float64[1])."""
        d = dims_of(x.shape)
        out = torch.empty(x.shape, dtype=torch.uint8, device=x.device) if out is None else out
        imax = torch.zeros(1, dtype=torch.float64, device=x.device)
        self._check(self.L.roix_normalize8(self.ctx, x.data_ptr(), _dtype_code(x), d,
                                           float(dark), out.data_ptr(), imax.data_ptr(),
                                           _stream(stream)))
        return out, imax

    def greedy(self, pixels: torch.Tensor, mask: torch.Tensor, shape, eabs: float,
               out: torch.Tensor | None = None, stream=None):
        """Sec. 4.2.3 over every row's retained pixels; returns (Q, n[1])."""
        d = dims_of(shape)
        out = torch.empty_like(pixels) if out is None else out
        n = torch.zeros(1, dtype=torch.uint64, device=pixels.device)
        self._check(self.L.roix_greedy_quantize(self.ctx, pixels.data_ptr(), mask.data_ptr(), d,
                                                float(eabs), out.data_ptr(), n.data_ptr(),
                                                _stream(stream)))
        return out, n

    def greedy_batch(self, items, eabs: float, outs=None, stream=None):
        """Sec. 4.2.3 over several images in one call: items = [(pixels, mask,
        shape), ...]; returns ([Q, ...], n[len(items)])."""
        dev = items[0][0].device if items else torch.device("cuda")
        outs = [torch.empty_like(p) for p, _, _ in items] if outs is None else outs
        n = torch.zeros(max(len(items), 1), dtype=torch.uint64, device=dev)
        arr = (GreedyItem * max(len(items), 1))()
        for k, ((p, m, shape), q) in enumerate(zip(items, outs)):
            arr[k] = GreedyItem(p.data_ptr(), m.data_ptr(), dims_of(shape), q.data_ptr(),
                                n.data_ptr() + 8 * k)
        self._check(self.L.roix_greedy_quantize_batch(self.ctx, len(items), arr, float(eabs),
                                                      _stream(stream)))
        return outs, n[:len(items)]

    def extract_roi_paper(self, img: torch.Tensor, stream=None):
        """Paper-mode ROI of a uint8 image (every 2D slice): mask words,
        pixel count [1] and the (t1, t2) thresholds per slice."""
        d = dims_of(img.shape)
        words = int(self.L.roix_mask_words(d))
        mask = torch.empty(max(words, 1), dtype=torch.int32, device=img.device)
        pop = torch.zeros(1, dtype=torch.uint64, device=img.device)
        thr = torch.zeros((max(int(d.nz), 1), 2), dtype=torch.int32, device=img.device)
        self._check(self.L.roix_extract_roi_paper(self.ctx, img.data_ptr(), d, mask.data_ptr(),
                                                  pop.data_ptr(), thr.data_ptr(),
                                                  _stream(stream)))
        return mask[:words], pop, thr

    def roi_quality(self, pred: torch.Tensor, truth: torch.Tensor, shape, distances=True,
                    stream=None) -> dict:
        """Sec. 5.2 metrics of mask words `pred` against `truth` (synchronises)."""
        out = torch.zeros(C.sizeof(RoiMetrics), dtype=torch.uint8, device=pred.device)
        self._check(self.L.roix_roi_quality(self.ctx, pred.data_ptr(), truth.data_ptr(),
                                            dims_of(shape), int(bool(distances)),
                                            out.data_ptr(), _stream(stream)))
        self.sync(stream)
        raw = bytes(out.cpu().numpy())
        m = RoiMetrics.from_buffer_copy(raw)
        return {k: getattr(m, k) for k, _ in RoiMetrics._fields_}

    def ssim(self, x: torch.Tensor, y: torch.Tensor, data_range: float, stream=None):
        """Sec. 5.6 mean SSIM of x and y; returns a float64 device tensor [1]."""
        out = torch.zeros(1, dtype=torch.float64, device=x.device)
        self._check(self.L.roix_ssim(self.ctx, x.data_ptr(), y.data_ptr(), _dtype_code(x),
                                     dims_of(x.shape), float(data_range), out.data_ptr(),
                                     _stream(stream)))
        return out

    def quantize(self, pixels: torch.Tensor, n_cap: int | None = None,
                 n_dev: torch.Tensor | None = None, stream=None, **cfg):
        n_cap = pixels.numel() if n_cap is None else n_cap
        dark = cfg.get("dark", 0.0)
        q = torch.empty(max(n_cap, 1), dtype=torch.int32, device=pixels.device)
        ob = torch.empty(max((n_cap + 31) // 32, 1), dtype=torch.int32, device=pixels.device)
        info = torch.zeros(C.sizeof(EbInfo), dtype=torch.uint8, device=pixels.device)
        self._check(self.L.roix_quantize(
            self.ctx, pixels.data_ptr(), _dtype_code(pixels), int(n_cap),
            n_dev.data_ptr() if n_dev is not None else None, C.byref(eb_of(**cfg)), float(dark),
            q.data_ptr(), ob.data_ptr(), info.data_ptr(), _stream(stream)))
        return q, ob, info

    def encode(self, q, obits, pixels, n_cap, sizes, counts, bounds, info, shape, dtype,
               cap: int | None = None, out: torch.Tensor | None = None, stream=None, **cfg):
        dev = q.device
        if out is None:
            cap = cap if cap is not None else self.bound(shape, dtype, **cfg)
            out = torch.empty(cap, dtype=torch.uint8, device=dev)
        cap = out.numel() if cap is None else cap
        size = torch.zeros(1, dtype=torch.uint64, device=dev)
        self._check(self.L.roix_encode(
            self.ctx, q.data_ptr(), obits.data_ptr(), pixels.data_ptr(), int(n_cap),
            sizes.data_ptr(), counts.data_ptr(), bounds.data_ptr(), info.data_ptr(),
            F32 if dtype == torch.float32 else U16, dims_of(shape), C.byref(roi_of(**cfg)),
            C.byref(eb_of(**cfg)), C.byref(params_of(**cfg)), out.data_ptr(), int(cap),
            size.data_ptr(), _stream(stream)))
        return out, size


class RoixServer:
    """Continuous-batching compression server on one GPU (roix_server_*).
    Inputs and outputs are caller-owned device tensors that must stay alive
    until their completion has been polled."""

    def __init__(self, device: int = 0, hbm_budget: int = 8 << 30, lanes: int = 4,
                 max_batch: int = 64):
        self.L = lib()
        h = C.c_void_p()
        cfg = ServerConfig(int(hbm_budget), int(lanes), int(max_batch))
        rc = self.L.roix_server_create(int(device), C.byref(cfg), C.byref(h))
        if rc != 0:
            raise RoixError(rc, "server create")
        self.h = h

    def submit(self, tag: int, x: torch.Tensor, out: torch.Tensor, cap: int | None = None,
               **cfg) -> int:
        """Returns the status (0 = queued)."""
        r = Request(int(tag), x.data_ptr(), _dtype_code(x), dims_of(x.shape), roi_of(**cfg),
                    eb_of(**cfg), params_of(**cfg), out.data_ptr(),
                    int(out.numel() if cap is None else cap))
        return int(self.L.roix_server_submit(self.h, C.byref(r)))

    def poll(self, max_n: int = 256):
        buf = (Completion * max_n)()
        k = self.L.roix_server_poll(self.h, buf, max_n)
        return [dict(tag=buf[i].tag, status=buf[i].status, size=buf[i].size,
                     t_submit=buf[i].t_submit, t_admit=buf[i].t_admit, t_done=buf[i].t_done)
                for i in range(k)]

    def drain(self, timeout_s: float = 60.0) -> int:
        return int(self.L.roix_server_drain(self.h, float(timeout_s)))

    def stats(self) -> dict:
        st = ServerStats()
        self.L.roix_server_get_stats(self.h, C.byref(st))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.L.roix_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
