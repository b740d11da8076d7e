"""Seeded synthetic X-CT inputs shaped like the paper's workloads.

This module is the one piece shared by the oracle side and the CUDA side: it
draws inputs and holds none of the compression method's arithmetic. The paper's
own datasets (Sec. 5, Table 1: wood, fossil embryos, Ryugu, chicken, walnut,
pine cone, seashell scans) are not available; these phantoms stand in for them:

* ``ellipsoids``       reconstructed volume: random rotated ellipsoids of
                       attenuation U(0.2, 1.0) in zero-valued air + Gaussian noise.
* ``projections``      flat-field uint16 projections: Poisson counts with open-beam
                       level I0, attenuated along parallel rays through a random
                       ellipsoid phantom, plus a constant dark offset (Sec. 4.1.1).
* ``porous_cylinder``  reconstructed volume: a cylinder of material with spherical
                       pores on zero-valued air, optional lognormal texture, noise.
* ``walk8``, ``runs``  8-bit rows that drift by small random steps (flat stretches
                       and slopes, as in a normalised image) and random run masks,
                       for the row-wise stages on their own.

Structure parameters come from ``numpy.random.default_rng(seed)``; per-voxel
noise and Poisson counts from a ``torch.Generator`` seeded with ``seed`` on the
device the volume is built on. Arrays are C-ordered (z, y, x): x is fastest.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-random 3x3 rotation (QR of a Gaussian matrix, signs fixed)."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _ellipsoid_params(rng, n, count, semi_lo, semi_hi):
    out = []
    for _ in range(count):
        c = rng.uniform(0.25, 0.75, size=3) * n
        a = rng.uniform(semi_lo, semi_hi, size=3) * (n / 128.0)
        rot = _rotation(rng)
        mu = rng.uniform(0.2, 1.0)
        out.append((c, a, rot, mu))
    return out


def ellipsoids(n: int = 128, count: int = 5, sigma: float = 0.01, seed: int = 0,
               device: str | torch.device = "cpu", shape=None) -> torch.Tensor:
    """n^3 float32 volume (or ``shape`` = (nz, ny, nx)); later ellipsoids overwrite
    earlier ones; air = 0; N(0, sigma^2) noise on every voxel."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape if shape is not None else (n, n, n)
    ref = min(nx, ny, nz)
    vol = torch.zeros((nz, ny, nx), dtype=torch.float32, device=device)
    for c, a, rot, mu in _ellipsoid_params(rng, ref, count, 8.0, 32.0):
        c = c * np.array([nx, ny, nz], dtype=np.float64) / ref
        # bounding box of the rotated ellipsoid
        ext = np.sqrt((rot ** 2) @ (a ** 2))
        lo = np.maximum(np.floor(c - ext).astype(int), 0)
        hi = np.minimum(np.ceil(c + ext).astype(int) + 1, [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        zs = torch.arange(lo[2], hi[2], device=device, dtype=torch.float64)
        ys = torch.arange(lo[1], hi[1], device=device, dtype=torch.float64)
        xs = torch.arange(lo[0], hi[0], device=device, dtype=torch.float64)
        Z, Y, X = torch.meshgrid(zs - c[2], ys - c[1], xs - c[0], indexing="ij")
        r = torch.as_tensor(rot.T / a[:, None], device=device)  # body coords / axes
        u = r[0, 0] * X + r[0, 1] * Y + r[0, 2] * Z
        v = r[1, 0] * X + r[1, 1] * Y + r[1, 2] * Z
        w = r[2, 0] * X + r[2, 1] * Y + r[2, 2] * Z
        inside = (u * u + v * v + w * w) <= 1.0
        sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        sub[inside] = float(mu)
    if sigma > 0:
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        vol += sigma * torch.randn(vol.shape, generator=g, device=device, dtype=torch.float32)
    return vol


def projection_sides(count: int = 64, lo: int = 512, hi: int = 2048, seed: int = 0):
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(lo, hi + 1, size=count)]


def projection(side: int, index: int, i0: float = 60000.0, dark: int = 100,
               max_path: float = 1.5, seed: int = 0,
               device: str | torch.device = "cpu") -> torch.Tensor:
    """One side x side uint16 projection: counts = Poisson(i0 * exp(-p)) + dark,
    clamped to 65535, with p the parallel-beam line integral (analytic chords)
    through a 5-ellipsoid phantom scaled to the detector, max p about max_path."""
    rng = np.random.default_rng([seed, index])
    ells = _ellipsoid_params(rng, side, 5, 8.0, 32.0)
    ys = torch.arange(side, device=device, dtype=torch.float64)
    Y, X = torch.meshgrid(ys, ys, indexing="ij")
    path = torch.zeros((side, side), dtype=torch.float64, device=device)
    for c, a, rot, mu in ells:
        # quadratic form M = R diag(1/a^2) R^T; ray (x, y, t) along z
        m = rot @ np.diag(1.0 / a ** 2) @ rot.T
        dx = X - c[0]
        dy = Y - c[1]
        qa = m[2, 2]
        qb = 2.0 * (m[0, 2] * dx + m[1, 2] * dy)
        qc = m[0, 0] * dx * dx + 2.0 * m[0, 1] * dx * dy + m[1, 1] * dy * dy - 1.0
        disc = (qb * qb - 4.0 * qa * qc).clamp_min(0.0)
        path += mu * torch.sqrt(disc) / qa
    peak = float(path.max())
    if peak > 0:
        path *= max_path / peak
    g = torch.Generator(device=device)
    g.manual_seed(seed * 1000003 + index)
    lam = (i0 * torch.exp(-path)).to(torch.float32)
    counts = torch.poisson(lam, generator=g) + float(dark)
    return counts.clamp_(0, 65535).to(torch.int32).to(torch.uint16)


def projections(count: int = 64, lo: int = 512, hi: int = 2048, seed: int = 0,
                device: str | torch.device = "cpu", **kw):
    return [projection(s, i, seed=seed, device=device, **kw)
            for i, s in enumerate(projection_sides(count, lo, hi, seed))]


def _smooth_1d(rng, n, device):
    """Unit-variance smooth sequence: sum of 4 random cosines."""
    t = torch.arange(n, device=device, dtype=torch.float64)
    s = torch.zeros(n, device=device, dtype=torch.float64)
    for _ in range(4):
        k = rng.uniform(1.0, 8.0) * 2.0 * math.pi / max(n, 1)
        s += math.sqrt(0.5) * torch.cos(k * t + rng.uniform(0, 2 * math.pi))
    return s


def porous_cylinder(n: int = 1024, radius: float = 400.0, fraction: float = 0.20,
                    pore_lo: float = 2.0, pore_hi: float = 30.0, porosity: float = 0.05,
                    sigma: float = 0.005, texture: bool = False, seed: int = 0,
                    z_range=None, device: str | torch.device = "cpu") -> torch.Tensor:
    """n^3 float32 volume: cylinder along z of the given radius, its height cut
    so that it fills ``fraction`` of the voxels, centred; value 1.0 (or the
    lognormal texture exp(0.25 (a[x] + b[y] + c[z]) / sqrt 3)); spherical pores
    of radius U(pore_lo, pore_hi) drawn uniformly inside the cylinder until their
    nominal volume reaches ``porosity`` of the cylinder; air 0; N(0, sigma^2).
    ``z_range`` = (z0, z1) builds only those slices (same values as the full
    volume there, noise included)."""
    rng = np.random.default_rng(seed)
    height = min(n, int(round(fraction * n ** 3 / (math.pi * radius ** 2))))
    z_lo = (n - height) // 2
    z_hi = z_lo + height
    cx = cy = (n - 1) / 2.0
    cyl_vol = math.pi * radius ** 2 * height
    pores = []
    acc = 0.0
    while acc < porosity * cyl_vol:
        r = rng.uniform(pore_lo, pore_hi)
        rho = radius * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        pz = rng.uniform(z_lo, z_hi)
        pores.append((cx + rho * math.cos(th), cy + rho * math.sin(th), pz, r))
        acc += 4.0 / 3.0 * math.pi * r ** 3
    tex = None
    if texture:
        tex = [_smooth_1d(rng, n, device) for _ in range(3)]
    z0, z1 = z_range if z_range is not None else (0, n)
    vol = torch.zeros((z1 - z0, n, n), dtype=torch.float32, device=device)
    ys = torch.arange(n, device=device, dtype=torch.float64)
    Y, X = torch.meshgrid(ys, ys, indexing="ij")
    disk = ((X - cx) ** 2 + (Y - cy) ** 2) <= radius ** 2
    a0, a1 = max(z0, z_lo), min(z1, z_hi)
    if a1 > a0:
        if tex is None:
            vol[a0 - z0:a1 - z0][:, disk] = 1.0
        else:
            base = (tex[0][None, :] + tex[1][:, None])  # (y, x)
            for z in range(a0, a1):
                val = torch.exp(0.25 * (base + tex[2][z]) / math.sqrt(3.0)).to(torch.float32)
                sl = vol[z - z0]
                sl[disk] = val[disk]
    for px, py, pz, r in pores:
        lo = [int(math.floor(px - r)), int(math.floor(py - r)), int(math.floor(pz - r))]
        hi = [int(math.ceil(px + r)) + 1, int(math.ceil(py + r)) + 1, int(math.ceil(pz + r)) + 1]
        lo = [max(lo[0], 0), max(lo[1], 0), max(lo[2], z0)]
        hi = [min(hi[0], n), min(hi[1], n), min(hi[2], z1)]
        if hi[0] <= lo[0] or hi[1] <= lo[1] or hi[2] <= lo[2]:
            continue
        zz = torch.arange(lo[2], hi[2], device=device, dtype=torch.float64) - pz
        yy = torch.arange(lo[1], hi[1], device=device, dtype=torch.float64) - py
        xx = torch.arange(lo[0], hi[0], device=device, dtype=torch.float64) - px
        d2 = zz[:, None, None] ** 2 + yy[None, :, None] ** 2 + xx[None, None, :] ** 2
        sub = vol[lo[2] - z0:hi[2] - z0, lo[1]:hi[1], lo[0]:hi[0]]
        sub[d2 <= r * r] = 0.0
    if sigma > 0:
        # noise drawn slice by slice from per-slice generators, so that a z_range
        # build reproduces the full volume's slices exactly
        g = torch.Generator(device=device)
        for z in range(z0, z1):
            g.manual_seed(seed * 1000003 + z)
            vol[z - z0] += sigma * torch.randn((n, n), generator=g, device=device,
                                               dtype=torch.float32)
    return vol


def random_field(shape, seed: int = 0, scale: float = 1.0, smooth: bool = True,
                 dtype=np.float32) -> np.ndarray:
    """Small test field: a smooth random walk along x (so that prediction has
    something to predict) or white noise; numpy, on the host."""
    rng = np.random.default_rng(seed)
    if smooth:
        steps = rng.standard_normal(shape) * scale * 0.05
        field = np.cumsum(steps, axis=-1) + rng.standard_normal(shape[:-1] + (1,)) * scale
    else:
        field = rng.standard_normal(shape) * scale
    return field.astype(dtype)


def walk8(shape, seed: int = 0, step: int = 3, hold: float = 0.3) -> np.ndarray:
    """uint8 image whose rows are clipped random walks from U[0, 255]: each
    pixel repeats the previous one with probability `hold`, else moves by
    U[-step, step]."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    nx = shape[-1]
    d = rng.integers(-step, step + 1, (rows, nx))
    d[rng.random((rows, nx)) < hold] = 0
    d[:, 0] = rng.integers(0, 256, rows)
    return np.clip(np.cumsum(d, axis=1), 0, 255).astype(np.uint8).reshape(shape)


def runs(shape, seed: int = 0, density: float = 0.5, mean_run: float = 40.0) -> np.ndarray:
    """uint8 0/1 mask whose rows alternate off/on runs of geometric lengths
    (mean `mean_run` when on)."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    nx = shape[-1]
    m = np.zeros((rows, nx), np.uint8)
    off_mean = mean_run * (1.0 - density) / max(density, 1e-6)
    for r in range(rows):
        x, on = 0, bool(rng.random() < density)
        while x < nx:
            length = int(rng.geometric(1.0 / max(mean_run if on else off_mean, 1.0)))
            if on:
                m[r, x:x + length] = 1
            x += length
            on = not on
    return m.reshape(shape)
