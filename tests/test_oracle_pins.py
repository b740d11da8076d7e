"""Pins of the CPU oracle against things other than itself: closed forms,
brute force on tiny inputs, independent library routines (scipy.ndimage,
numpy indexing, heapq Huffman), invariants and textbook values."""
from __future__ import annotations

import heapq
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import phantom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ndimage = pytest.importorskip("scipy.ndimage")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ threshold
def test_threshold_golden_edges():
    rows = _load("threshold_edges.txt")
    x = np.array([int(r[0], 16) for r in rows], np.uint32).view(np.float32)
    gt = oracle.threshold(x, cmp="gt", threshold=0.1)
    lt = oracle.threshold(x, cmp="lt", threshold=0.1)
    assert gt.tolist() == [int(r[1]) for r in rows]
    assert lt.tolist() == [int(r[2]) for r in rows]


def test_threshold_uint16_dark_subtraction():
    # Sec. 4.1.1: M = I - B with B = dark; object where M < 57000 (config of the
    # flat-field projections). Integers, so the comparison is exact.
    raw = np.array([0, 100, 57099, 57100, 57101, 65535], np.uint16)
    T = oracle.threshold(raw, cmp="lt", threshold=57000, dark=100)
    assert T.tolist() == [1, 1, 1, 0, 0, 0]
    T = oracle.threshold(raw, cmp="gt", threshold=0.5, dark=100)
    assert T.tolist() == [0, 0, 1, 1, 1, 1]


# ------------------------------------------------------------------- dilation
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 7, 9), (5, 6, 7), (9, 4, 33)])
@pytest.mark.parametrize("density", [0.02, 0.2])
def test_dilation_matches_scipy(shape, density):
    rng = np.random.default_rng(hash((shape, density)) % 2**32)
    T = (rng.random(shape) < density).astype(np.uint8)
    D = oracle.dilate(T, 1)
    ref = ndimage.binary_dilation(T.astype(bool), structure=np.ones((3, 3, 3), bool))
    assert np.array_equal(D.astype(bool), ref)
    assert np.array_equal(oracle.dilate(T, 0), T)


def test_dilation_2d_is_3x3():
    T = np.zeros((1, 5, 5), np.uint8)
    T[0, 2, 2] = 1
    D = oracle.dilate(T, 1)
    assert D.sum() == 9 and D[0, 1:4, 1:4].all()


# --------------------------------------------------------- largest component
@pytest.mark.parametrize("conn", [6, 26])
@pytest.mark.parametrize("seed", range(6))
def test_keep_largest_matches_scipy_label(conn, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(rng.integers(4, 12, size=3))
    T = (rng.random(shape) < rng.uniform(0.2, 0.6)).astype(np.uint8)
    st = ndimage.generate_binary_structure(3, 1 if conn == 6 else 3)
    lab, nlab = ndimage.label(T, structure=st)
    got = oracle.keep_largest(T, conn)
    if nlab == 0:
        assert got.sum() == 0
        return
    sizes = np.bincount(lab.ravel())[1:]
    best = sizes.max()
    # tie: component containing the smallest raster index
    cands = [c + 1 for c in range(nlab) if sizes[c] == best]
    first = {c: np.flatnonzero(lab.ravel() == c)[0] for c in cands}
    keep = min(cands, key=lambda c: first[c])
    assert np.array_equal(got.astype(bool), lab == keep)


def test_keep_largest_tie_goes_to_first():
    T = np.zeros((1, 3, 7), np.uint8)
    T[0, 0, 0:2] = 1  # size 2, first
    T[0, 2, 5:7] = 1  # size 2, later
    got = oracle.keep_largest(T, 26)
    assert got[0, 0, 0:2].all() and got.sum() == 2


def test_connectivity_diagonal():
    T = np.zeros((1, 3, 3), np.uint8)
    T[0, 0, 0] = T[0, 1, 1] = T[0, 2, 2] = 1  # one 8-connected line
    assert oracle.keep_largest(T, 26).sum() == 3
    assert oracle.keep_largest(T, 6).sum() == 1


# ----------------------------------------------------------------- compaction
@pytest.mark.parametrize("shape", [(3, 5, 31), (2, 4, 64), (1, 1, 1), (4, 3, 70)])
def test_compaction_is_boolean_indexing_and_runs_rebuild_mask(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape).astype(np.float32)
    D = (rng.random(shape) < 0.4).astype(np.uint8)
    P, counts, bounds = oracle.compact(x, D)
    assert np.array_equal(P, x[D.astype(bool)])
    # rebuild the mask from the run boundaries (x_start, x_end pairs)
    nz, ny, nx = shape
    rebuilt = np.zeros(shape, bool)
    b = 0
    for r in range(ny * nz):
        c = int(counts[r])
        assert c % 2 == 0
        for i in range(0, c, 2):
            xs, xe = int(bounds[b + i]), int(bounds[b + i + 1])
            assert 0 <= xs < xe <= nx
            rebuilt[r // ny, r % ny, xs:xe] = True
        b += c
    assert b == bounds.size
    assert np.array_equal(rebuilt, D.astype(bool))


def test_compaction_full_row_boundaries():
    x = np.arange(6, dtype=np.float32).reshape(1, 1, 6)
    P, counts, bounds = oracle.compact(x, np.ones((1, 1, 6), np.uint8))
    assert counts.tolist() == [2] and bounds.tolist() == [0, 6]
    assert P.tolist() == list(range(6))


# ------------------------------------------------------------------- quantiser
def _exact_err(x, q, two_eb):
    return abs(Fraction(float(x)) - Fraction(float(np.float32(np.float32(q) * np.float32(two_eb)))))


@pytest.mark.parametrize("eb", [1e-3, 0.05, 0.5, 3.0, 1e-6])
def test_quantize_error_bound_and_nearest_lattice_point(eb):
    rng = np.random.default_rng(int(eb * 1e6) % 1000)
    x = np.concatenate([
        rng.standard_normal(400).astype(np.float32),
        (rng.integers(-50, 50, 100) * np.float32(2 * eb) + np.float32(eb)).astype(np.float32),
        np.array([0.0, -0.0, np.float32(eb), -np.float32(eb)], np.float32)])
    e = oracle.error_bound(x, "abs", eb)
    q, o = oracle.quantize(x, e)
    ebq = Fraction(eb)
    for xi, qi, oi in zip(x, q, o):
        if oi:
            assert qi == 0
            # an outlier is a value the binary32 lattice cannot hold within E_abs:
            # it sits within a few ulps of a cell edge (half-way between points)
            t = Fraction(float(xi)) * Fraction(float(e.inv2eb))
            dist = abs(t - round(t))
            ulps = Fraction(float(np.spacing(np.abs(xi)))) * Fraction(float(e.inv2eb))
            assert dist >= Fraction(1, 2) - (abs(t) / 2**22 + 4 * ulps)
            continue
        # the decoder's value differs from x by at most E_abs (Sec. 4.2.3), exactly
        assert _exact_err(xi, qi, e.two_eb) <= ebq
        # nearest lattice point, up to the rounding of one binary32 product
        # (half an ulp of the product: |t| 2^-24, doubled for the comparison)
        t = Fraction(float(xi)) * Fraction(float(e.inv2eb))
        slack = abs(t) / 2**23 + Fraction(1, 2**140)
        for cand in (qi - 1, qi + 1):
            assert abs(t - qi) <= abs(t - cand) + slack
    # generic values are almost never outliers while the lattice is fine enough
    if eb >= 1e-3:
        assert o[:400].sum() <= 2


def test_quantize_exact_multiples_power_of_two_step():
    # 2 E_abs = 2^-4: every multiple of 2^-4 is a lattice point, q = x * 16 exactly
    eb = 2.0 ** -5
    k = np.arange(-1000, 1000)
    x = (k / 16.0).astype(np.float32)
    e = oracle.error_bound(x, "abs", eb)
    q, o = oracle.quantize(x, e)
    assert not o.any() and np.array_equal(q, k)


def test_quantize_cell_edges_are_kept_verbatim():
    # lattice step 1: a half-integer lies exactly E_abs from two lattice points;
    # the check keeps a margin below E_abs, so such values are outliers, while a
    # value one ulp inside the cell is coded
    eb = 0.5
    x = np.array([0.5, 1.5, -2.5, np.nextafter(np.float32(1.5), np.float32(0))], np.float32)
    q, o = oracle.quantize(x, oracle.error_bound(x, "abs", eb))
    assert o.tolist() == [1, 1, 1, 0] and q.tolist() == [0, 0, 0, 1]


def test_quantize_outliers():
    x = np.array([np.nan, np.inf, -np.inf, 3e38, 1.0], np.float32)
    e = oracle.error_bound(x, "abs", 1e-3)
    q, o = oracle.quantize(x, e)
    assert o.tolist() == [1, 1, 1, 1, 0] and q[:4].tolist() == [0, 0, 0, 0]
    # a bound too small for binary32 makes every value an outlier (kept verbatim)
    e = oracle.error_bound(x, "abs", 1e-45)
    q, o = oracle.quantize(x, e)
    assert o.all()


def test_relative_bound_uses_finite_range_of_retained_values():
    x = np.array([np.nan, -2.0, 6.0, np.inf, 1.0], np.float32)
    e = oracle.error_bound(x, "rel", 1e-2)
    assert e.vmin == -2.0 and e.vmax == 6.0 and e.eb_abs == pytest.approx(0.08)
    e = oracle.error_bound(np.array([3.0, 3.0], np.float32), "rel", 1e-2)
    assert e.eb_abs == 0.0 and e.bound < 0  # zero range: lossless fallback


@pytest.mark.parametrize("eb", [0, 1, 4, 7])
def test_quantize_uint16_brute_force(eb):
    raw = np.arange(0, 2000, dtype=np.uint16)
    dark = 100
    e = oracle.error_bound(raw, "abs", eb)
    q, o = oracle.quantize(raw, e, dark=dark)
    assert not o.any()
    for r, qi in zip(raw.tolist(), q.tolist()):
        v = r - dark
        if eb == 0:
            assert qi == v
            continue
        ok = [c for c in range(v // (2 * eb) - 3, v // (2 * eb) + 4) if abs(v - 2 * eb * c) <= eb]
        assert qi == max(ok)  # within the bound; the upper lattice point on a tie


# ------------------------------------------------------------------ prediction
def _inverse_lorenzo(sym, rk, rv, R):
    """Independent inverse: prefix sum of the deltas, records override."""
    rec = {int(k) & ((1 << 63) - 1): (int(k) >> 63, int(v)) for k, v in zip(rk, rv)}
    out, prev = [], 0
    for k, s in enumerate(sym.tolist()):
        if s:
            c = prev + s - R
        else:
            kind, v = rec[k]
            c = 0 if kind else int(np.array(v, np.uint32).view(np.int32))
        out.append(c)
        prev = c
    return np.array(out, np.int64)


@pytest.mark.parametrize("R", [2, 16, 512])
def test_lorenzo_inverts_and_records_sit_on_symbol_zero(R):
    rng = np.random.default_rng(R)
    q = np.cumsum(rng.integers(-3 * R, 3 * R, 500)).astype(np.int32)
    outl = (rng.random(500) < 0.05).astype(np.uint8)
    q[outl.astype(bool)] = 0
    P = rng.standard_normal(500).astype(np.float32)
    sym, rk, rv = oracle.lorenzo(q, outl, P, R)
    assert np.array_equal(_inverse_lorenzo(sym, rk, rv, R), q.astype(np.int64))
    keys = rk & np.uint64((1 << 63) - 1)
    assert np.array_equal(keys, np.flatnonzero(sym == 0).astype(np.uint64))
    assert (sym < 2 * R).all()
    kinds = (rk >> np.uint64(63)).astype(bool)
    assert np.array_equal(np.flatnonzero(outl), keys[kinds].astype(np.int64))
    assert np.array_equal(rv[kinds], P[outl.astype(bool)].view(np.uint32))


def _inverse_lorenzo2(sym, rk, rv, R):
    """Independent inverse of the two-layer Lorenzo: c = 2 c[k-1] - c[k-2] + d."""
    rec = {int(k) & ((1 << 63) - 1): (int(k) >> 63, int(v)) for k, v in zip(rk, rv)}
    out, p1, p2 = [], 0, 0
    for k, s in enumerate(sym.tolist()):
        if s:
            c = 2 * p1 - p2 + s - R
        else:
            kind, v = rec[k]
            c = 0 if kind else int(np.array(v, np.uint32).view(np.int32))
        out.append(c)
        p2, p1 = p1, c
    return np.array(out, np.int64)


@pytest.mark.parametrize("R", [2, 16, 512])
def test_lorenzo2_inverts_and_records_sit_on_symbol_zero(R):
    rng = np.random.default_rng(R + 7)
    q = np.cumsum(np.cumsum(rng.integers(-R, R, 500))).astype(np.int32)
    outl = (rng.random(500) < 0.05).astype(np.uint8)
    q[outl.astype(bool)] = 0
    P = rng.standard_normal(500).astype(np.float32)
    sym, rk, rv = oracle.lorenzo(q, outl, P, R, order=2)
    assert np.array_equal(_inverse_lorenzo2(sym, rk, rv, R), q.astype(np.int64))
    keys = rk & np.uint64((1 << 63) - 1)
    assert np.array_equal(keys, np.flatnonzero(sym == 0).astype(np.uint64))
    kinds = (rk >> np.uint64(63)).astype(bool)
    assert np.array_equal(np.flatnonzero(outl), keys[kinds].astype(np.int64))


def test_lorenzo2_closed_forms():
    # second differences of a quadratic are constant (2a); of a line, zero; the
    # first two residuals are q0 and q1 - 2 q0 (q[-1] = q[-2] = 0)
    R = 512
    k = np.arange(300, dtype=np.int64)
    for a, b, c0 in [(1, -3, 7), (-2, 40, -100), (0, 5, 11)]:
        q = (a * k * k + b * k + c0).astype(np.int32)
        z = np.zeros(q.size, np.uint8)
        P = np.zeros(q.size, np.float32)
        sym, rk, rv = oracle.lorenzo(q, z, P, R, order=2)
        assert (sym[2:].astype(np.int64) == 2 * a + R).all()
        assert int(sym[0]) == c0 + R and int(sym[1]) == (a + b + c0) - 2 * c0 + R
        assert rk.size == 0
        # order 1 on the same line: constant first difference b (a = 0 case)
        if a == 0:
            s1, _, _ = oracle.lorenzo(q, z, P, R, order=1)
            assert (s1[1:].astype(np.int64) == b + R).all()


@pytest.mark.parametrize("cfg", [dict(eb=1e-3, eb_mode="abs"), dict(eb=1e-4, eb_mode="rel"),
                                 dict(eb=1e-5, eb_mode="rel", radius=16)])
def test_predictor_changes_the_stream_not_the_values(cfg):
    # the codes are the same under either predictor, so the decoded values are
    # bit-identical; only the symbols (and the size) differ
    x = phantom.porous_cylinder(40, radius=15, texture=True, seed=4).numpy()
    b1 = oracle.compress(x, predictor=1, **cfg)
    b2 = oracle.compress(x, predictor=2, **cfg)
    assert oracle.header(b1)["order"] == 1 and oracle.header(b2)["order"] == 2
    y1 = oracle.decode(b1, x.shape, np.float32)
    y2 = oracle.decode(b2, x.shape, np.float32)
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))
    D = oracle.mask(x, **cfg).astype(bool)
    assert _exact_within(x[D], y2[D], oracle.header(b2)["eb_abs"])


def test_histogram_is_bincount():
    sym = np.random.default_rng(1).integers(0, 64, 1000).astype(np.uint16)
    assert np.array_equal(oracle.histogram(sym, 64), np.bincount(sym, minlength=64))


# -------------------------------------------------------------------- codebook
def _heap_huffman_cost(freqs):
    h = [int(f) for f in freqs if f > 0]
    if len(h) < 2:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def _check_canonical_prefix_code(ln, cd):
    syms = [s for s in range(ln.size) if ln[s]]
    words = sorted((int(ln[s]), s, format(int(cd[s]), f"0{int(ln[s])}b")) for s in syms)
    for i in range(len(words) - 1):
        a, b = words[i][2], words[i + 1][2]
        assert not b.startswith(a)
        # canonical: consecutive codes in (length, symbol) order increase by one
        assert int(b, 2) == (int(a, 2) + 1) << (len(b) - len(a))
    assert words[0][2] == "0" * words[0][0]


def test_codebook_textbook_example():
    rows = _load("huffman_textbook.txt")
    h = np.zeros(8, np.uint64)
    for s, f, _ in rows:
        h[int(s)] = int(f)
    ln, cd = oracle.codebook(h)
    assert [int(ln[int(s)]) for s, _, _ in rows] == [int(r[2]) for r in rows]
    assert int((h * ln).sum()) == 224
    _check_canonical_prefix_code(ln, cd)


@pytest.mark.parametrize("seed", range(8))
def test_codebook_optimal_kraft_canonical(seed):
    rng = np.random.default_rng(seed)
    S = int(rng.choice([4, 32, 1024]))
    h = (rng.geometric(rng.uniform(0.01, 0.5), S) * (rng.random(S) < 0.7)).astype(np.uint64)
    h[rng.integers(0, S)] += 1  # at least one symbol
    ln, cd = oracle.codebook(h)
    used = h > 0
    assert np.array_equal(ln > 0, used)
    if used.sum() >= 2:
        assert sum(Fraction(1, 2 ** int(l)) for l in ln[used]) == 1
        assert int((h * ln.astype(np.uint64)).sum()) == _heap_huffman_cost(h)
        _check_canonical_prefix_code(ln, cd)
    else:
        assert ln[used].tolist() == [1]


def test_codebook_length_limit_on_fibonacci_counts():
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    h = np.array(fib, np.uint64)  # unconstrained Huffman depth would be 39
    ln, cd = oracle.codebook(h)
    assert ln.max() == 24 and (ln > 0).all()
    assert sum(Fraction(1, 2 ** int(l)) for l in ln) == 1
    _check_canonical_prefix_code(ln, cd)
    # more frequent never gets a longer code
    order = np.argsort(h, kind="stable")
    assert all(ln[order[i]] >= ln[order[i + 1]] for i in range(len(order) - 1))


def test_codebook_degenerate():
    ln, _ = oracle.codebook(np.zeros(16, np.uint64))
    assert not ln.any()
    h = np.zeros(16, np.uint64)
    h[5] = 10
    ln, cd = oracle.codebook(h)
    assert ln[5] == 1 and ln.sum() == 1 and cd[5] == 0


# ------------------------------------------------------------------------ pack
def _unpack(off, words, ln, cd, n, chunk):
    table = {(int(ln[s]), int(cd[s])): s for s in range(ln.size) if ln[s]}
    bits = np.unpackbits(words.astype(">u4").view(np.uint8))  # MSB-first per word
    out = []
    for j, w0 in enumerate(off.tolist()):
        p = 32 * w0
        for _ in range(min(chunk, n - j * chunk)):
            l, c = 0, 0
            while (l, c) not in table:
                c = (c << 1) | int(bits[p])
                p += 1
                l += 1
                assert l <= 24
            out.append(table[(l, c)])
    return np.array(out, np.uint16)


@pytest.mark.parametrize("n,chunk", [(0, 256), (1, 256), (1000, 256), (5000, 4096), (4096, 4096)])
def test_pack_unpacks_with_independent_bit_reader(n, chunk):
    rng = np.random.default_rng(n)
    sym = np.minimum(rng.geometric(0.2, n), 63).astype(np.uint16)
    h = oracle.histogram(sym, 64)
    ln, cd = oracle.codebook(h)
    off, words = oracle.pack(sym, ln, cd, chunk)
    assert off.size == (n + chunk - 1) // chunk
    if n:
        assert off[0] == 0 and (np.diff(off.astype(np.int64)) >= 0).all()
        total_bits = int((h * ln.astype(np.uint64)).sum())
        assert 32 * words.size >= total_bits
    assert np.array_equal(_unpack(off, words, ln, cd, n, chunk), sym)


# ------------------------------------------------------------ whole container
def _exact_within(x, xh, eb):
    xd = x.astype(np.float64)
    hd = xh.astype(np.float64)
    return np.all(np.abs(xd - hd) <= eb)


@pytest.mark.parametrize("eb", [1e-3, 1e-2])
def test_container_round_trip_float32_ellipsoids(eb):
    x = phantom.ellipsoids(40, seed=3).numpy()
    cfg = dict(eb=eb, threshold=0.1, dilate=1)
    buf = oracle.compress(x, **cfg)
    hdr = oracle.header(buf)
    D = oracle.mask(x, **cfg).astype(bool)
    assert hdr["magic"] == b"ROIX" and hdr["total"] == buf.size
    assert hdr["n"] == D.sum() and 0 < hdr["n"] < x.size
    y = oracle.decode(buf, x.shape, np.float32)
    # Sec. 4.2.3 bound on every retained voxel, checked in binary64 (exact here:
    # the difference of two nearby binary32 values is representable)
    assert _exact_within(x[D], y[D], eb)
    assert (y[~D] == 0).all()
    assert buf.size < x.nbytes  # it compresses


def test_container_round_trip_uint16_projection():
    x = phantom.projection(96, 0).numpy()
    cfg = dict(eb=4, eb_mode="abs", cmp="lt", threshold=57000, dark=100, dilate=0,
               fill=60100)
    buf = oracle.compress(x, **cfg)
    D = oracle.mask(x, **cfg).astype(bool)
    y = oracle.decode(buf, x.shape, np.uint16)
    assert np.abs(x[D].astype(np.int64) - y[D].astype(np.int64)).max() <= 4
    assert (y[~D] == 60100).all()


def test_container_lossless_uint16_and_outliers_float32():
    x = phantom.projection(64, 1).numpy()
    cfg = dict(eb=0, cmp="lt", threshold=57000, dark=100, dilate=0, fill=0)
    y = oracle.decode(oracle.compress(x, **cfg), x.shape, np.uint16)
    D = oracle.mask(x, **cfg).astype(bool)
    assert np.array_equal(y[D], x[D])
    # float32 with non-finite values and huge magnitudes: kept verbatim
    f = phantom.random_field((3, 5, 37), seed=2)
    f[0, 0, :5] = [np.nan, np.inf, -np.inf, 3e38, -3e38]
    # NaN and -inf never pass the threshold; the dilation retains them
    buf = oracle.compress(f, eb=1e-3, cmp="gt", threshold=-1e30, dilate=1)
    assert oracle.header(buf)["n"] == f.size
    y = oracle.decode(buf, f.shape, np.float32)
    assert np.array_equal(y[0, 0, :5].view(np.uint32), f[0, 0, :5].view(np.uint32))
    fin = np.isfinite(f) & (np.abs(f) < 1e30)
    assert _exact_within(f[fin], y[fin], 1e-3)
    assert oracle.header(buf)["n_outliers"] >= 5


def test_container_relative_bound():
    x = phantom.porous_cylinder(48, radius=18, seed=1).numpy()
    cfg = dict(eb=1e-3, eb_mode="rel", threshold=0.1, dilate=1)
    buf = oracle.compress(x, **cfg)
    D = oracle.mask(x, **cfg).astype(bool)
    rng_ = float(x[D].max()) - float(x[D].min())
    hdr = oracle.header(buf)
    assert hdr["eb_abs"] == pytest.approx(1e-3 * rng_, rel=1e-12)
    y = oracle.decode(buf, x.shape, np.float32)
    assert _exact_within(x[D], y[D], hdr["eb_abs"])


def test_container_edge_shapes():
    for shape in [(1, 1, 1), (2, 3, 1), (1, 1, 70), (3, 2, 65)]:
        x = phantom.random_field(shape, seed=len(shape))
        for thr in (-1e9, 1e9):  # everything, nothing
            buf = oracle.compress(x, eb=1e-2, threshold=thr, dilate=1)
            y = oracle.decode(buf, shape, np.float32)
            if thr < 0:
                assert _exact_within(x, y, 1e-2)
            else:
                assert oracle.header(buf)["n"] == 0 and (y == 0).all()
    x = np.zeros((0, 4, 4), np.float32)
    buf = oracle.compress(x, eb=1e-2)
    assert oracle.header(buf)["n"] == 0


def test_keep_largest_in_container():
    x = np.zeros((1, 12, 12), np.float32)
    x[0, 1:3, 1:3] = 1.0   # 4 voxels
    x[0, 6:10, 6:10] = 1.0  # 16 voxels: kept
    buf = oracle.compress(x, eb=1e-3, threshold=0.5, keep="largest", dilate=0)
    y = oracle.decode(buf, x.shape, np.float32)
    assert (y[0, 6:10, 6:10] == 1.0).all() and y.sum() == 16


def test_decode_rejects_corruption():
    x = phantom.random_field((2, 4, 40), seed=9)
    buf = oracle.compress(x, eb=1e-2, threshold=-1e9)
    with pytest.raises(ValueError):
        oracle.decode(buf[:100], x.shape, np.float32)
    bad = buf.copy()
    bad[0] = ord("X")
    with pytest.raises(ValueError):
        oracle.decode(bad, x.shape, np.float32)
    with pytest.raises(ValueError):
        oracle.decode(buf, (2, 4, 41), np.float32)
    with pytest.raises(ValueError):
        oracle.decode(buf[:-64], x.shape, np.float32)


# ----------------------------------- 8-bit normalisation + greedy quantiser
def _min_groups_brute(D, e):
    """Minimum number of constant groups with |Q - D| <= e (integers), by
    dynamic programming over all segmentations (independent of the greedy)."""
    m = len(D)
    best = [0] + [10**9] * m
    for j in range(1, m + 1):
        for i in range(j):
            lo = max(int(d) - e for d in D[i:j])
            hi = min(int(d) + e for d in D[i:j])
            if lo <= hi:
                best[j] = min(best[j], best[i] + 1)
    return best[m]


def _groups(Q):
    return 0 if len(Q) == 0 else 1 + int(np.count_nonzero(np.diff(Q.astype(np.int64))))


def test_greedy_hand_example():
    # D = 1 2 3 10, E = 1: [0,2] n [1,3] n [2,4] = [2,2] -> 2 2 2; then [9,11] -> 10
    assert oracle.greedy_seq(np.array([1, 2, 3, 10], np.uint8), 1).tolist() == [2, 2, 2, 10]
    # odd u + l rounds down: [0,2] n [1,3] = [1,2] -> floor(3/2) = 1
    assert oracle.greedy_seq(np.array([1, 2], np.uint8), 1).tolist() == [1, 1]
    # touching ranges still overlap: [-1,1] n [1,3] = [1,1]
    assert oracle.greedy_seq(np.array([0, 2], np.uint8), 1).tolist() == [1, 1]
    assert oracle.greedy_seq(np.array([0, 3], np.uint8), 1).tolist() == [0, 3]
    # E < 1 keeps every value: groups are runs of equal pixels
    D = np.array([5, 5, 6, 200, 200, 0], np.uint8)
    assert np.array_equal(oracle.greedy_seq(D, 0.1), D)


@pytest.mark.parametrize("seed", range(12))
def test_greedy_bound_and_minimal_groups(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 14))
    D = np.clip(np.cumsum(rng.integers(-6, 7, m)) + 128, 0, 255).astype(np.uint8)
    for e in (0, 1, 2, 5, 15):
        Q = oracle.greedy_seq(D, e + 0.5 * (seed % 2))  # fractional E uses floor(E)
        assert (np.abs(Q.astype(int) - D.astype(int)) <= e).all()
        # constant groups: the greedy closes a group only when it must, so it
        # reaches the minimum number of groups (interval stabbing)
        assert _groups(Q) <= _min_groups_brute(D, e)


def test_greedy_clips_to_8_bits():
    D = np.array([255, 254, 0, 1], np.uint8)
    Q = oracle.greedy_seq(D, 15)
    assert Q.max() <= 255 and (np.abs(Q.astype(int) - D.astype(int)) <= 15).all()


def test_normalize8_closed_form_points():
    x = np.array([0.0, 1.0, 2.0, 4.0, -3.0, np.nan, 0.5], np.float32)
    img, imax = oracle.normalize8(x)
    assert imax == 4.0
    # 4 -> 255; 2 -> 127.5 -> 128 (half to even); 1 -> 63.75 -> 64; 0.5 -> 31.875 -> 32
    assert img.tolist() == [0, 64, 128, 255, 0, 0, 32]
    raw = np.array([100, 100, 355, 610], np.uint16)  # v = 0, 0, 255, 510
    img, imax = oracle.normalize8(raw, dark=100)
    assert imax == 510.0 and img.tolist() == [0, 0, 128, 255]


def test_greedy_rows_resets_per_row():
    img = np.array([[10, 11, 12, 50], [12, 13, 90, 91]], np.uint8)
    mask = np.array([[1, 1, 1, 0], [1, 1, 1, 1]], np.uint8)
    # row 0: [9,11] n [10,12] n [11,13] = [11,11]; row 1 starts afresh:
    # [11,13] n [12,14] = [12,13] -> 12, then [89,91] n [90,92] = [90,91] -> 90
    assert oracle.greedy_rows(img, mask, 1).tolist() == [11, 11, 11, 12, 12, 90, 90]


def test_normalize8_u16_exact_rational_half_even():
    from fractions import Fraction
    rng = np.random.default_rng(3)
    raw = rng.integers(0, 4000, 3000).astype(np.uint16)
    raw[:4] = [0, 37, 2037, 3999]
    img, imax = oracle.normalize8(raw, dark=37)
    v = np.maximum(raw.astype(np.int64) - 37, 0)
    assert imax == v.max()
    want = [round(Fraction(255 * int(a), int(imax))) for a in v]  # Python rounds half to even
    assert img.tolist() == want


def test_normalize8_f32_error_and_order():
    rng = np.random.default_rng(4)
    x = rng.gamma(2.0, 1.5, 20000).astype(np.float32)
    x[::97] = -x[::97]
    x[5] = np.inf
    img, imax = oracle.normalize8(x)
    v = np.where(np.isfinite(x) & (x > 0), x, 0).astype(np.float64)
    assert imax == v.max()
    exact = v / imax * 255.0
    # two binary32 roundings then rounding to an integer: within 1/2 + a few ulps
    assert np.abs(img - exact).max() <= 0.5 + 1e-4
    order = np.argsort(v, kind="stable")
    assert (np.diff(img[order].astype(int)) >= 0).all()  # monotone in v
    assert img[np.argmax(v)] == 255 and (img[v == 0] == 0).all()


def test_normalize8_zero_image():
    img, imax = oracle.normalize8(np.zeros(10, np.uint16), dark=0)
    assert imax == 0 and not img.any()
    img, imax = oracle.normalize8(np.full(10, -1.0, np.float32))
    assert imax == 0 and not img.any()


def test_uint8_threshold_and_compact():
    rng = np.random.default_rng(6)
    img = rng.integers(0, 256, (3, 7, 45)).astype(np.uint8)
    T = oracle.threshold(img, threshold=140.5, cmp="gt", dilate=0)
    assert np.array_equal(T, (img > 140.5).astype(np.uint8))
    T = oracle.threshold(img, threshold=20, cmp="lt", dark=5, dilate=0)
    assert np.array_equal(T, (img.astype(int) - 5 < 20).astype(np.uint8))
    P, counts, bounds = oracle.compact(img, T)
    assert np.array_equal(P, img[T.astype(bool)])


def test_uint8_refused_by_linear_path():
    with pytest.raises(Exception):
        oracle.compress(np.zeros((4, 4), np.uint8))


# --------------------------------------------------------------- z-slabs
@pytest.mark.parametrize("cfg", [dict(eb=1e-3, eb_mode="abs", dilate=1),
                                 dict(eb=1e-3, eb_mode="rel", dilate=1),
                                 dict(eb=1e-2, eb_mode="rel", dilate=0)])
def test_slabs_decode_like_the_whole_volume(cfg):
    x = phantom.ellipsoids(shape=(21, 18, 23), seed=8).numpy()
    whole = oracle.compress(x, **cfg)
    want = oracle.decode(whole, x.shape, np.float32)
    for slab_z in (1, 4, 7, 21, 40):
        conts = oracle.compress_slabs(x, slab_z, **cfg)
        assert len(conts) == -(-21 // slab_z)
        got = np.concatenate([oracle.decode(c, (oracle.header(c)["nz"],) + x.shape[1:], np.float32)
                              for c in conts])
        # the dilation crosses slab borders and the bound is the volume's: the
        # decoded values equal the whole-volume decode voxel for voxel
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), slab_z
        assert sum(oracle.header(c)["n"] for c in conts) == oracle.header(whole)["n"]
        assert all(oracle.header(c)["eb_abs"] == oracle.header(whole)["eb_abs"] for c in conts)
    assert np.array_equal(oracle.compress_slabs(x, 21, **cfg)[0], whole)


@pytest.mark.parametrize("cfg", [dict(eb=1e-3, eb_mode="rel", dilate=1),
                                 dict(eb=1e-3, eb_mode="abs", dilate=0)])
def test_slab_from_its_slices_and_halo_equals_the_slabbed_volume(cfg):
    # a slab encoded from its own slices plus one neighbouring slice on each
    # side and the volume's error bound equals that slab of compress_slabs, and
    # the slabs' decodes stacked equal the whole-volume decode
    x = phantom.ellipsoids(shape=(22, 17, 29), seed=12).numpy()
    D = oracle.mask(x, **cfg)
    P, _, _ = oracle.compact(x, D)
    e = oracle.error_bound(P, cfg["eb_mode"], cfg["eb"])
    whole = oracle.decode(oracle.compress(x, **cfg), x.shape, np.float32)
    for slab_z in (1, 5, 22):
        conts = oracle.compress_slabs(x, slab_z, **cfg)
        dec = []
        for k, z0 in enumerate(range(0, 22, slab_z)):
            dz = min(slab_z, 22 - z0)
            h0, h1 = max(0, z0 - 1), min(22, z0 + dz + 1)
            got = oracle.encode_slab(x[h0:h1], z0 - h0, dz, e, **cfg)
            assert np.array_equal(got, conts[k]), (slab_z, k)
            dec.append(oracle.decode(got, (dz,) + x.shape[1:], np.float32))
        assert np.array_equal(np.concatenate(dec).view(np.uint32), whole.view(np.uint32))
    with pytest.raises(RuntimeError):  # more than one halo slice after the slab
        oracle.encode_slab(x[0:5], 0, 3, e, **cfg)


def test_slabs_refuse_keep():
    x = phantom.ellipsoids(shape=(8, 8, 8), seed=1).numpy()
    with pytest.raises(RuntimeError):
        oracle.compress_slabs(x, 4, keep="largest")
