"""CPU oracle for the ROIX-Comp hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``roix_oracle.cpp`` (plain,
single-threaded C++17 compiled with ``-O2 -ffp-contract=off``) through ctypes and
shares nothing with the CUDA library: not its header, its parameter structs or
its binding. Arrays are numpy, C-ordered (z, y, x) with x fastest.

Section references are to the paper (ROIX-Comp, arXiv 2602.15917); each stage
function names the step it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "roix_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, U16, U8 = 1, 2, 3
HEADER_BYTES = 256
LMAX = 24


def build(force: bool = False) -> str:
    """Compile the oracle (g++, no fast-math, no FP contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


class _Params(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("eb_mode", C.c_int32), ("eb_value", C.c_double),
                ("cmp", C.c_int32), ("keep", C.c_int32), ("connectivity", C.c_int32),
                ("dilate", C.c_int32), ("threshold", C.c_double), ("dark", C.c_double),
                ("fill", C.c_double), ("radius", C.c_uint32), ("chunk", C.c_uint32),
                ("order", C.c_uint32)]


class Eb(C.Structure):
    _fields_ = [("eb_abs", C.c_double), ("vmin", C.c_double), ("vmax", C.c_double),
                ("two_eb", C.c_float), ("inv2eb", C.c_float), ("bound", C.c_float),
                ("eb_int", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_OUT)
            P, u64, i32, u32, d = C.c_void_p, C.c_uint64, C.c_int32, C.c_uint32, C.c_double
            L.oracle_threshold.argtypes = [P, C.POINTER(_Params), u64, u64, u64, P]
            L.oracle_keep_largest.argtypes = [P, u64, u64, u64, i32]
            L.oracle_dilate.argtypes = [P, u64, u64, u64, i32, P]
            L.oracle_compact.argtypes = [P, i32, u64, u64, u64, P, P, P, P, P]
            L.oracle_compact.restype = C.c_int64
            L.oracle_eb.argtypes = [P, i32, u64, i32, d, C.POINTER(Eb)]
            L.oracle_eb.restype = None
            L.oracle_quantize.argtypes = [P, i32, u64, C.POINTER(Eb), d, P, P]
            L.oracle_lorenzo.argtypes = [P, P, P, i32, u64, u32, u32, P, P, P]
            L.oracle_lorenzo.restype = u64
            L.oracle_histogram.argtypes = [P, u64, u32, P]
            L.oracle_histogram.restype = None
            L.oracle_codebook.argtypes = [P, u32, P, P]
            L.oracle_pack.argtypes = [P, u64, P, P, u32, P, P]
            L.oracle_pack.restype = u64
            L.oracle_compress.argtypes = [P, C.POINTER(_Params), u64, u64, u64,
                                          C.POINTER(C.c_void_p), C.POINTER(u64)]
            L.oracle_compress_slabs.argtypes = [P, C.POINTER(_Params), u64, u64, u64, u64,
                                                C.POINTER(C.c_void_p), C.POINTER(u64)]
            L.oracle_encode_slab.argtypes = [P, C.POINTER(_Params), u64, u64, u64, u64, u64,
                                             C.POINTER(Eb), C.POINTER(C.c_void_p),
                                             C.POINTER(u64)]
            L.oracle_free.argtypes = [P]
            L.oracle_free.restype = None
            L.oracle_decode.argtypes = [P, u64, P, i32, u64, u64, u64]
            L.oracle_normalize8.argtypes = [P, i32, u64, d, P]
            L.oracle_normalize8.restype = d
            L.oracle_greedy_seq.argtypes = [P, u64, d, P]
            L.oracle_greedy_seq.restype = None
            L.oracle_greedy_rows.argtypes = [P, P, u64, u64, u64, d, P]
            L.oracle_greedy_rows.restype = u64
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(x: np.ndarray):
    if x.ndim == 2:
        return x.shape[1], x.shape[0], 1
    if x.ndim == 3:
        return x.shape[2], x.shape[1], x.shape[0]
    if x.ndim == 1:
        return x.shape[0], 1, 1
    raise ValueError("1D, 2D or 3D arrays only")


def _dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return F32
    if x.dtype == np.uint16:
        return U16
    if x.dtype == np.uint8:
        return U8
    raise TypeError("float32, uint16 or uint8 input")


def params(dtype: int, eb=1e-3, eb_mode="abs", cmp="gt", threshold=0.1, keep="all",
           connectivity=26, dilate=1, dark=0.0, fill=0.0, radius=512, chunk=4096,
           predictor=1) -> _Params:
    return _Params(dtype, 0 if eb_mode == "abs" else 1, float(eb), 0 if cmp == "gt" else 1,
                   0 if keep == "all" else 1, int(connectivity), int(dilate),
                   float(threshold), float(dark), float(fill), int(radius), int(chunk),
                   int(predictor))


# ------------------------------------------------------------------- stages
def threshold(x: np.ndarray, **cfg) -> np.ndarray:
    """Sec. 4.1.1 + 4.1.3-4.1.4: binary mask T (uint8, same shape)."""
    x = np.ascontiguousarray(x)
    p = params(_dtype_code(x), **cfg)
    T = np.zeros(x.shape, np.uint8)
    lib().oracle_threshold(_ptr(x), C.byref(p), *_dims(x), _ptr(T))
    return T


def keep_largest(T: np.ndarray, connectivity: int = 26) -> np.ndarray:
    """Sec. 4.2.1: the largest connected component (flood fill)."""
    T = np.ascontiguousarray(T, dtype=np.uint8).copy()
    lib().oracle_keep_largest(_ptr(T), *_dims(T), int(connectivity))
    return T


def dilate(T: np.ndarray, radius: int = 1) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.uint8)
    D = np.zeros_like(T)
    lib().oracle_dilate(_ptr(T), *_dims(T), int(radius), _ptr(D))
    return D


def mask(x: np.ndarray, **cfg) -> np.ndarray:
    """threshold -> (largest component) -> dilation: the retained-voxel mask D."""
    T = threshold(x, **cfg)
    if cfg.get("keep", "all") != "all":
        T = keep_largest(T, cfg.get("connectivity", 26))
    return dilate(T, cfg.get("dilate", 1))


def compact(x: np.ndarray, D: np.ndarray):
    """Sec. 4.2.2: pixel section P (ROI values in raster order), per-row
    boundary counts and the boundary list (x_start, x_end pairs)."""
    x = np.ascontiguousarray(x)
    D = np.ascontiguousarray(D, dtype=np.uint8)
    nx, ny, nz = _dims(x)
    rows = ny * nz
    P = np.zeros(max(x.size, 1), x.dtype)
    counts = np.zeros(max(rows, 1), np.uint16)
    bounds = np.zeros(max(rows * (nx + 1), 1), np.uint16)
    nb = C.c_uint64(0)
    n = lib().oracle_compact(_ptr(x), _dtype_code(x), nx, ny, nz, _ptr(D), _ptr(P),
                             _ptr(counts), _ptr(bounds), C.byref(nb))
    return P[:n].copy(), counts[:rows].copy(), bounds[:nb.value].copy()


def error_bound(P: np.ndarray, eb_mode="abs", eb=1e-3) -> Eb:
    P = np.ascontiguousarray(P)
    e = Eb()
    lib().oracle_eb(_ptr(P), _dtype_code(P), P.size, 0 if eb_mode == "abs" else 1,
                    float(eb), C.byref(e))
    return e


def quantize(P: np.ndarray, e: Eb, dark: float = 0.0):
    """Sec. 4.2.3 contract |Q - D| <= E_abs: codes q and outlier flags."""
    P = np.ascontiguousarray(P)
    q = np.zeros(max(P.size, 1), np.int32)
    o = np.zeros(max(P.size, 1), np.uint8)
    lib().oracle_quantize(_ptr(P), _dtype_code(P), P.size, C.byref(e), float(dark),
                          _ptr(q), _ptr(o))
    return q[:P.size].copy(), o[:P.size].copy()


def lorenzo(q: np.ndarray, outl: np.ndarray, P: np.ndarray, radius: int = 512, order: int = 1):
    """1D Lorenzo prediction of the given order (1, or 2 for the two-layer form)
    + symbols; returns (sym, record keys, record payloads)."""
    n = q.size
    q = np.ascontiguousarray(q, np.int32)
    outl = np.ascontiguousarray(outl, np.uint8)
    P = np.ascontiguousarray(P)
    sym = np.zeros(max(n, 1), np.uint16)
    rk = np.zeros(max(n, 1), np.uint64)
    rv = np.zeros(max(n, 1), np.uint32)
    m = lib().oracle_lorenzo(_ptr(q), _ptr(outl), _ptr(P), _dtype_code(P), n, int(radius),
                             int(order), _ptr(sym), _ptr(rk), _ptr(rv))
    return sym[:n].copy(), rk[:m].copy(), rv[:m].copy()


def histogram(sym: np.ndarray, nsym: int) -> np.ndarray:
    sym = np.ascontiguousarray(sym, np.uint16)
    h = np.zeros(nsym, np.uint64)
    lib().oracle_histogram(_ptr(sym), sym.size, int(nsym), _ptr(h))
    return h


def codebook(hist: np.ndarray):
    """Canonical, length-limited Huffman code: (lengths uint8, codes uint32)."""
    hist = np.ascontiguousarray(hist, np.uint64)
    ln = np.zeros(hist.size, np.uint8)
    cd = np.zeros(hist.size, np.uint32)
    lib().oracle_codebook(_ptr(hist), hist.size, _ptr(ln), _ptr(cd))
    return ln, cd


def pack(sym: np.ndarray, lengths: np.ndarray, codes: np.ndarray, chunk: int = 4096):
    """Chunked MSB-first bit packing: (chunk word offsets, payload words)."""
    sym = np.ascontiguousarray(sym, np.uint16)
    nch = (sym.size + chunk - 1) // chunk
    off = np.zeros(max(nch, 1), np.uint64)
    L = lib()
    nw = L.oracle_pack(_ptr(sym), sym.size, _ptr(lengths), _ptr(codes), int(chunk), _ptr(off), None)
    words = np.zeros(max(nw, 1), np.uint32)
    L.oracle_pack(_ptr(sym), sym.size, _ptr(lengths), _ptr(codes), int(chunk), _ptr(off), _ptr(words))
    return off[:nch].copy(), words[:nw].copy()


# -------------------------------------------------------------- whole path
def compress(x: np.ndarray, **cfg) -> np.ndarray:
    """The whole compression path; returns the container bytes (uint8)."""
    x = np.ascontiguousarray(x)
    p = params(_dtype_code(x), **cfg)
    out = C.c_void_p()
    size = C.c_uint64(0)
    L = lib()
    rc = L.oracle_compress(_ptr(x), C.byref(p), *_dims(x), C.byref(out), C.byref(size))
    if rc != 0:
        raise RuntimeError(f"oracle_compress failed ({rc})")
    try:
        buf = np.ctypeslib.as_array(C.cast(out, C.POINTER(C.c_uint8)), shape=(size.value,)).copy()
    finally:
        L.oracle_free(out)
    return buf


def compress_slabs(x: np.ndarray, slab_z: int, **cfg):
    """A volume in z-slabs of slab_z slices, one container per slab (the mask
    and the error bound are the whole volume's); returns a list of uint8 arrays."""
    x = np.ascontiguousarray(x)
    p = params(_dtype_code(x), **cfg)
    nx, ny, nz = _dims(x)
    ns = (nz + slab_z - 1) // slab_z
    outs = (C.c_void_p * max(ns, 1))()
    sizes = (C.c_uint64 * max(ns, 1))()
    L = lib()
    rc = L.oracle_compress_slabs(_ptr(x), C.byref(p), nx, ny, nz, int(slab_z), outs, sizes)
    res = []
    try:
        if rc != 0:
            raise RuntimeError(f"oracle_compress_slabs failed ({rc})")
        for k in range(ns):
            res.append(np.ctypeslib.as_array(C.cast(outs[k], C.POINTER(C.c_uint8)),
                                             shape=(sizes[k],)).copy())
    finally:
        for k in range(ns):
            if outs[k]:
                L.oracle_free(outs[k])
    return res


def encode_slab(xbuf: np.ndarray, z0: int, dz: int, e: Eb, **cfg) -> np.ndarray:
    """One z-slab's container from its slices alone: xbuf holds the slab's dz
    slices starting at slice z0 (0 or 1) with the volume's neighbouring slice
    on each side where the volume has one; e = the whole volume's error-bound
    constants. Equals that slab's container of compress_slabs."""
    xbuf = np.ascontiguousarray(xbuf)
    p = params(_dtype_code(xbuf), **cfg)
    nx, ny, nzb = _dims(xbuf)
    out = C.c_void_p()
    size = C.c_uint64(0)
    L = lib()
    rc = L.oracle_encode_slab(_ptr(xbuf), C.byref(p), nx, ny, nzb, int(z0), int(dz),
                              C.byref(e), C.byref(out), C.byref(size))
    if rc != 0:
        raise RuntimeError(f"oracle_encode_slab failed ({rc})")
    try:
        buf = np.ctypeslib.as_array(C.cast(out, C.POINTER(C.c_uint8)), shape=(size.value,)).copy()
    finally:
        L.oracle_free(out)
    return buf


def decode(buf: np.ndarray, shape, dtype) -> np.ndarray:
    """Sec. 4.3 reconstruction; raises ValueError on a corrupt container."""
    buf = np.ascontiguousarray(buf, np.uint8)
    out = np.zeros(shape, dtype)
    rc = lib().oracle_decode(_ptr(buf), buf.size, _ptr(out), _dtype_code(out), *_dims(out))
    if rc != 0:
        raise ValueError(f"corrupt container ({rc})")
    return out


def header(buf: np.ndarray) -> dict:
    """Named header fields of a container (little-endian, fixed offsets)."""
    b = bytes(np.ascontiguousarray(buf, np.uint8)[:HEADER_BYTES])
    f = lambda off, t: np.frombuffer(b, t, 1, off)[0].item()
    return dict(magic=b[:4], version=f(4, "<u2"), dtype=b[6], eb_mode=b[7],
                nx=f(8, "<u4"), ny=f(12, "<u4"), nz=f(16, "<u4"), cmp=b[20], keep=b[21],
                connectivity=b[22], dilate=b[23], threshold=f(24, "<f8"), dark=f(32, "<f8"),
                fill=f(40, "<f8"), eb_value=f(48, "<f8"), eb_abs=f(56, "<f8"),
                two_eb=f(64, "<f4"), inv2eb=f(68, "<f4"), bound=f(72, "<f4"),
                eb_int=f(76, "<i4"), radius=f(80, "<u4"), chunk=f(84, "<u4"),
                lmax=f(88, "<u4"), order=max(1, f(92, "<u4")), n=f(96, "<u8"), n_outliers=f(104, "<u8"),
                n_bounds=f(112, "<u8"), n_chunks=f(120, "<u8"), payload_words=f(128, "<u8"),
                vmin=f(136, "<f8"), vmax=f(144, "<f8"), off_lens=f(152, "<u8"),
                off_counts=f(160, "<u8"), off_bounds=f(168, "<u8"), off_outk=f(176, "<u8"),
                off_outv=f(184, "<u8"), off_chunks=f(192, "<u8"), off_payload=f(200, "<u8"),
                total=f(208, "<u8"))


# ------------------------------------------ the paper's 8-bit quantiser path
def normalize8(x: np.ndarray, dark: float = 0.0):
    """Sec. 4.1.2: 8-bit image I_n = round(v / I_max * 255); returns (I_n, I_max)."""
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint8:
        raise TypeError("float32 or uint16 input")
    out = np.zeros(x.shape, np.uint8)
    imax = lib().oracle_normalize8(_ptr(x), _dtype_code(x), x.size, float(dark), _ptr(out))
    return out, imax


def greedy_seq(D: np.ndarray, eabs: float) -> np.ndarray:
    """Sec. 4.2.3 on one sequence of 8-bit pixels."""
    D = np.ascontiguousarray(D, np.uint8)
    Q = np.zeros(max(D.size, 1), np.uint8)
    lib().oracle_greedy_seq(_ptr(D), D.size, float(eabs), _ptr(Q))
    return Q[:D.size].copy()


def greedy_rows(img: np.ndarray, mask: np.ndarray, eabs: float) -> np.ndarray:
    """Quantised pixel section: every row's retained pixels as one sequence."""
    img = np.ascontiguousarray(img, np.uint8)
    mask = np.ascontiguousarray(mask, np.uint8)
    Q = np.zeros(max(img.size, 1), np.uint8)
    n = lib().oracle_greedy_rows(_ptr(img), _ptr(mask), *_dims(img), float(eabs), _ptr(Q))
    return Q[:n].copy()
