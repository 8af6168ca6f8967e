"""Seeded synthetic vessel-network volumes and initial level sets.

These stand in for the paper's micro-CT, light-sheet and knife-edge / milling
microscopy data (Sec. 5.2), which are not available.  The module holds input
generation only -- no step of the level-set method -- and is the one module
shared by the product tests, the benchmark and the oracle tests.

Recipe (every volume): a branching random walk lays down capsule segments
(segment length U[6, 20] voxels, direction jitter <= 40 degrees per segment,
branch probability 0.3, radius uniform in the workload's range); each capsule
is rasterised with partial-volume occupancy clip(r - d + 0.5, 0, 1), where d
is the distance of the voxel centre from the segment, and capsules are
max-composited (so the order does not matter); the occupancy is blurred by a
separable Gaussian point-spread function, mapped to intensity
background + (foreground - background) * occupancy, given noise, clipped and
rounded to the storage type.  Random streams are numpy PCG64 seeded with
1000 * workload + brick.

Arrays are numpy [nz, ny, nx] (x fastest), the layout of the C-ABI.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import os

import numpy as np

try:  # the point-spread blur and the box mean; scipy is present on both machines
    from scipy import ndimage as _ndi
except Exception:  # pragma: no cover
    _ndi = None


def rng_for(workload: int, brick: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * int(workload) + int(brick)))


# --------------------------------------------------------------- segments

def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v)


def _random_dir(rng: np.random.Generator) -> np.ndarray:
    return _unit(rng.normal(size=3))


def _jitter(rng: np.random.Generator, d: np.ndarray, max_deg: float, min_deg: float = 0.0) -> np.ndarray:
    """Rotate unit vector d by an angle in [min_deg, max_deg] about a random perpendicular axis."""
    a = np.deg2rad(rng.uniform(min_deg, max_deg))
    p = rng.normal(size=3)
    p -= p.dot(d) * d
    p = _unit(p)
    return _unit(np.cos(a) * d + np.sin(a) * p)


@dataclass
class Segments:
    """Capsules: endpoints p0, p1 (n, 3) in (x, y, z) voxel units and radii r (n,)."""
    p0: np.ndarray
    p1: np.ndarray
    r: np.ndarray

    def __len__(self) -> int:
        return int(self.r.shape[0])


def vessel_segments(rng: np.random.Generator, extent_xyz: Tuple[float, float, float], n_segments: int,
                    r_range: Tuple[float, float], seg_len=(6.0, 20.0), jitter_deg: float = 40.0,
                    p_branch: float = 0.3) -> Segments:
    """Branching random walk inside the box [0, extent) (x, y, z)."""
    ext = np.asarray(extent_xyz, dtype=np.float64)
    p0s, p1s, rs = [], [], []
    stack = []
    while len(rs) < n_segments:
        if not stack:
            stack.append((rng.uniform(0.0, 1.0, size=3) * ext, _random_dir(rng),
                          rng.uniform(r_range[0], r_range[1])))
        p, d, r = stack.pop()
        q = p + rng.uniform(seg_len[0], seg_len[1]) * d
        p0s.append(p)
        p1s.append(q)
        rs.append(r)
        if np.all(q >= -2.0) and np.all(q <= ext + 2.0):
            if rng.random() < p_branch:
                rb = float(np.clip(r * rng.uniform(0.6, 1.0), r_range[0], r_range[1]))
                stack.insert(0, (q, _jitter(rng, d, 90.0, 30.0), rb))
            stack.append((q, _jitter(rng, d, jitter_deg), r))
    return Segments(np.array(p0s), np.array(p1s), np.array(rs))


def rasterize(seg: Segments, origin_xyz, shape_zyx) -> np.ndarray:
    """Partial-volume occupancy of the box [origin, origin + shape) (float32, [z, y, x])."""
    oz, oy, ox = (int(origin_xyz[2]), int(origin_xyz[1]), int(origin_xyz[0]))
    nz, ny, nx = (int(s) for s in shape_zyx)
    occ = np.zeros((nz, ny, nx), dtype=np.float32)
    lo = np.minimum(seg.p0, seg.p1) - seg.r[:, None] - 1.0
    hi = np.maximum(seg.p0, seg.p1) + seg.r[:, None] + 1.0
    org = np.array([ox, oy, oz], dtype=np.float64)
    top = org + np.array([nx, ny, nz], dtype=np.float64)
    hit = np.all(hi >= org, axis=1) & np.all(lo <= top - 1, axis=1)
    for i in np.nonzero(hit)[0]:
        a = np.maximum(np.floor(lo[i]).astype(np.int64), org.astype(np.int64))
        b = np.minimum(np.ceil(hi[i]).astype(np.int64) + 1, top.astype(np.int64))
        if np.any(b <= a):
            continue
        xs = np.arange(a[0], b[0], dtype=np.float64)
        ys = np.arange(a[1], b[1], dtype=np.float64)
        zs = np.arange(a[2], b[2], dtype=np.float64)
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        p, q, r = seg.p0[i], seg.p1[i], seg.r[i]
        v = q - p
        vv = max(float(v.dot(v)), 1e-12)
        t = np.clip(((X - p[0]) * v[0] + (Y - p[1]) * v[1] + (Z - p[2]) * v[2]) / vv, 0.0, 1.0)
        dx = X - (p[0] + t * v[0])
        dy = Y - (p[1] + t * v[1])
        dz = Z - (p[2] + t * v[2])
        o = np.clip(r - np.sqrt(dx * dx + dy * dy + dz * dz) + 0.5, 0.0, 1.0).astype(np.float32)
        sl = (slice(a[2] - oz, b[2] - oz), slice(a[1] - oy, b[1] - oy), slice(a[0] - ox, b[0] - ox))
        np.maximum(occ[sl], o, out=occ[sl])
    return occ


def _blur(occ: np.ndarray, sig_zyx) -> np.ndarray:
    if _ndi is None:
        raise RuntimeError("scipy.ndimage is required for the point-spread blur")
    return _ndi.gaussian_filter(occ, sigma=sig_zyx, mode="reflect", truncate=3.0).astype(np.float32)


# ------------------------------------------------------------ workloads

@dataclass
class RSFParams:
    sigma: float = 3.0
    eps: float = 1.0
    lambda1: float = 1.0
    lambda2: float = 2.0
    nu: float = 0.004 * 255.0 ** 2
    mu: float = 1.0
    dt: float = 0.1
    iters: int = 50
    c0: float = 2.0

    def as_dict(self) -> dict:
        return dict(sigma=self.sigma, eps=self.eps, lambda1=self.lambda1, lambda2=self.lambda2,
                    nu=self.nu, mu=self.mu, dt=self.dt)


def box_phi0(shape_zyx, box: int, c0: float = 2.0) -> np.ndarray:
    """+c0 inside a centred box of edge `box`, -c0 elsewhere (float32)."""
    phi = np.full(shape_zyx, -c0, dtype=np.float32)
    sl = tuple(slice((n - box) // 2, (n - box) // 2 + box) for n in shape_zyx)
    phi[sl] = c0
    return phi


def mean_rule_phi0(vol: np.ndarray, c0: float = 2.0, slab: int = 64) -> np.ndarray:
    """+c0 where the 3x3x3 box mean of the image (clamped borders) exceeds the image mean.

    Computed slab by slab along z (each slab with its neighbouring planes), so
    that large volumes need no full-size float64 copy."""
    if _ndi is None:
        raise RuntimeError("scipy.ndimage is required for the box mean")
    nz = vol.shape[0]
    mean = float(np.mean(vol, dtype=np.float64))
    out = np.empty(vol.shape, dtype=np.float32)
    for z0 in range(0, nz, slab):
        z1 = min(z0 + slab, nz)
        a, b = max(z0 - 1, 0), min(z1 + 1, nz)
        m = _ndi.uniform_filter(vol[a:b].astype(np.float64), size=3, mode="nearest")[z0 - a:z0 - a + (z1 - z0)]
        out[z0:z1] = np.where(m > mean, c0, -c0)
    return out


def tree_volume_u8(shape_zyx=(64, 64, 64), workload: int = 1, brick: int = 0, n_segments: int = 40,
                   r_range=(1.0, 4.0), fg: float = 200.0, bg: float = 30.0, psf: float = 1.0,
                   noise: float = 15.0) -> np.ndarray:
    """Small uint8 vessel tree (the 64^3 parity workload)."""
    rng = rng_for(workload, brick)
    nz, ny, nx = shape_zyx
    seg = vessel_segments(rng, (nx, ny, nz), n_segments, r_range)
    occ = _blur(rasterize(seg, (0, 0, 0), shape_zyx), (psf, psf, psf))
    img = bg + (fg - bg) * occ + rng.normal(0.0, noise, size=occ.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def lightsheet_volume_u16(shape_zyx=(512, 512, 512), workload: int = 2, brick: int = 0,
                          n_segments: Optional[int] = None, r_range=(0.5, 3.0), peak: float = 4000.0,
                          background: float = 300.0, psf_xy: float = 1.0, psf_z: float = 2.5,
                          truth: bool = False):
    """uint16 light-sheet-like volume: anisotropic PSF and Poisson shot noise.

    ~2000 segments per 512^3; smaller shapes scale the count with the volume.
    With `truth`, also returns the ground-truth vessel mask: voxels whose
    partial-volume occupancy (before the point-spread blur) is at least 1/2.
    """
    rng = rng_for(workload, brick)
    nz, ny, nx = shape_zyx
    if n_segments is None:
        n_segments = max(8, int(round(2000 * (nz * ny * nx) / 512 ** 3)))
    seg = vessel_segments(rng, (nx, ny, nz), n_segments, r_range)
    occ0 = rasterize(seg, (0, 0, 0), shape_zyx)
    mask = occ0 >= 0.5 if truth else None
    occ = _blur(occ0, (psf_z, psf_xy, psf_xy))
    del occ0
    lam = background + peak * occ
    img = np.clip(rng.poisson(lam), 0, 65535).astype(np.uint16)
    return (img, mask) if truth else img


# ----------------------------------------------------- batched bricks

@dataclass
class BrickSpec:
    origin_xyz: Tuple[int, int, int]
    core_xyz: Tuple[int, int, int]
    halo: int

    @property
    def padded_zyx(self) -> Tuple[int, int, int]:
        cx, cy, cz = self.core_xyz
        h = 2 * self.halo
        return (cz + h, cy + h, cx + h)


@dataclass
class MicroCTField:
    """A virtual uint16 micro-CT-like volume rasterised only where bricks are requested."""
    extent_xyz: Tuple[int, int, int] = (2048, 2048, 1024)
    workload: int = 3
    r_range: Tuple[float, float] = (1.0, 6.0)
    fg: float = 1200.0
    bg: float = 400.0
    noise: float = 80.0
    psf: float = 1.0
    density: float = 2000.0 / 512 ** 3   # segments per voxel, as the light-sheet volume
    seg: Segments = field(init=False)

    def __post_init__(self):
        rng = rng_for(self.workload, 0)
        ex, ey, ez = self.extent_xyz
        n = int(self.density * ex * ey * ez)
        self.seg = vessel_segments(rng, (ex, ey, ez), n, self.r_range)

    def brick(self, spec: BrickSpec, brick_index: int) -> np.ndarray:
        """The padded brick (halo voxels included) as uint16 [z, y, x]."""
        m = int(np.ceil(3 * self.psf)) + 1
        nz, ny, nx = spec.padded_zyx
        ox, oy, oz = (o - spec.halo - m for o in spec.origin_xyz)
        occ = rasterize(self.seg, (ox, oy, oz), (nz + 2 * m, ny + 2 * m, nx + 2 * m))
        occ = _blur(occ, (self.psf,) * 3)[m:m + nz, m:m + ny, m:m + nx]
        rng = rng_for(self.workload, 1 + brick_index)
        img = self.bg + (self.fg - self.bg) * occ + rng.normal(0.0, self.noise, size=occ.shape)
        return np.clip(np.rint(img), 0, 65535).astype(np.uint16)


def brick_specs(n_bricks: int = 256, core_range=(64, 192), halo: int = 12,
                extent_xyz=(2048, 2048, 1024), workload: int = 3) -> list:
    """Uneven, non-cubic brick cores drawn U[core_range] per axis at random positions."""
    rng = rng_for(workload, 100000)
    out = []
    for _ in range(n_bricks):
        core = tuple(int(c) for c in rng.integers(core_range[0], core_range[1] + 1, size=3))
        org = tuple(int(rng.integers(halo, e - c - halo)) for e, c in zip(extent_xyz, core))
        out.append(BrickSpec(org, core, halo))
    return out


def milling_volume_u8(shape_zyx, workload: int = 4, brick: int = 0, vessel_fraction: float = 0.04,
                      r_range=(1.0, 2.0), fg: float = 200.0, bg: float = 30.0, stripe: float = 0.2,
                      stripe_period: float = 64.0, noise: float = 20.0, psf: float = 1.0) -> np.ndarray:
    """uint8 milling-microscopy-like volume: a dense capillary bed (radius 1-2 voxels,
    about 4 % vessel fraction), illumination striped by +-20 % along z (period 64
    voxels, a reading: the period is not given), Gaussian noise std 20."""
    rng = rng_for(workload, brick)
    nz, ny, nx = shape_zyx
    mean_len, mean_r = 13.0, 0.5 * (r_range[0] + r_range[1])
    n_seg = max(4, int(vessel_fraction * nx * ny * nz / (np.pi * mean_r ** 2 * mean_len)))
    seg = vessel_segments(rng, (nx, ny, nz), n_seg, r_range)
    occ = _blur(rasterize(seg, (0, 0, 0), shape_zyx), (psf, psf, psf))
    z = np.arange(nz, dtype=np.float32)[:, None, None]
    gain = 1.0 + stripe * np.sin(2.0 * np.pi * z / stripe_period)
    img = (bg + (fg - bg) * occ) * gain + rng.normal(0.0, noise, size=occ.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


@dataclass
class MillingField:
    """A uint8 milling-microscopy-like volume (dense capillary bed, radius 1-2
    voxels, about 4 % vessel fraction, illumination striped by +-20 % along z
    with period 64, Gaussian noise std 20), defined voxel by voxel so that any
    box of it is rasterised on its own and equals that region of the whole:
    segments are drawn once over the extent, occupancy is rasterised with a
    margin for the point-spread blur, and noise is drawn per global z plane."""
    extent_xyz: Tuple[int, int, int] = (1024, 1024, 1024)
    workload: int = 4
    vessel_fraction: float = 0.04
    r_range: Tuple[float, float] = (1.0, 2.0)
    fg: float = 200.0
    bg: float = 30.0
    stripe: float = 0.2
    stripe_period: float = 64.0
    noise: float = 20.0
    psf: float = 1.0
    seg: Segments = field(init=False)

    def __post_init__(self):
        ex, ey, ez = self.extent_xyz
        mean_len, mean_r = 13.0, 0.5 * (self.r_range[0] + self.r_range[1])
        n = max(4, int(self.vessel_fraction * ex * ey * ez / (np.pi * mean_r ** 2 * mean_len)))
        self.seg = vessel_segments(rng_for(self.workload, 0), (ex, ey, ez), n, self.r_range)

    def _plane_noise(self, z: int) -> np.ndarray:
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([1000 * self.workload, 7, int(z)])))
        ex, ey, _ = self.extent_xyz
        return rng.normal(0.0, self.noise, size=(ey, ex))

    def box(self, origin_xyz, shape_zyx) -> np.ndarray:
        """uint8 [z, y, x] of the box at origin (x, y, z) with shape (nz, ny, nx)."""
        m = int(np.ceil(3 * self.psf)) + 1
        nz, ny, nx = (int(v) for v in shape_zyx)
        ox, oy, oz = (int(v) for v in origin_xyz)
        occ = rasterize(self.seg, (ox - m, oy - m, oz - m), (nz + 2 * m, ny + 2 * m, nx + 2 * m))
        occ = _blur(occ, (self.psf,) * 3)[m:m + nz, m:m + ny, m:m + nx]
        z = (oz + np.arange(nz, dtype=np.float64))[:, None, None]
        img = (self.bg + (self.fg - self.bg) * occ) * (1.0 + self.stripe * np.sin(2.0 * np.pi * z / self.stripe_period))
        for i in range(nz):
            img[i] += self._plane_noise(oz + i)[oy:oy + ny, ox:ox + nx]
        return np.clip(np.rint(img), 0, 255).astype(np.uint8)


_FIELD_FOR_WORKER = None


def _field_worker_init(f):
    global _FIELD_FOR_WORKER
    _FIELD_FOR_WORKER = f


def _field_worker(job):
    z0, nzs = job
    ex, ey, _ = _FIELD_FOR_WORKER.extent_xyz
    return z0, _FIELD_FOR_WORKER.box((0, 0, z0), (nzs, ey, ex))


def field_volume(f: "MillingField", slab: int = 64, workers: Optional[int] = None) -> np.ndarray:
    """The whole volume of a box-rasterised field, slabs of `slab` planes built by a
    spawn-context process pool (safe after CUDA initialisation in the parent)."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context
    ex, ey, ez = f.extent_xyz
    jobs = [(z0, min(slab, ez - z0)) for z0 in range(0, ez, slab)]
    workers = workers or max(1, min(16, os.cpu_count() or 1, len(jobs)))
    if workers == 1:
        return np.concatenate([f.box((0, 0, z0), (n, ey, ex)) for z0, n in jobs])
    with ProcessPoolExecutor(max_workers=workers, mp_context=get_context("spawn"),
                             initializer=_field_worker_init, initargs=(f,)) as pool:
        parts = sorted(pool.map(_field_worker, jobs))
    return np.concatenate([v for _, v in parts])


@dataclass
class ServeRequestSpec:
    source: str          # "lightsheet", "microct" or "milling"
    core_zyx: Tuple[int, int, int]
    sigma: float
    iters: int

    @property
    def halo(self) -> int:
        return int(round(3 * self.sigma))

    @property
    def padded_zyx(self) -> Tuple[int, int, int]:
        return tuple(c + 2 * self.halo for c in self.core_zyx)


def serve_request_specs(n: int, workload: int = 5, core_range=(32, 256), sigmas=(2.0, 3.0, 4.0, 6.0),
                        iters_range=(50, 500)):
    """Request mix: core edges log-uniform in core_range per axis, sigma uniform in
    `sigmas`, iterations uniform in iters_range, data source uniform over the three."""
    rng = rng_for(workload, 0)
    lo, hi = np.log(core_range[0]), np.log(core_range[1])
    out = []
    for _ in range(n):
        core = tuple(int(round(np.exp(rng.uniform(lo, hi)))) for _ in range(3))
        out.append(ServeRequestSpec(str(rng.choice(["lightsheet", "microct", "milling"])), core,
                                    float(rng.choice(sigmas)), int(rng.integers(iters_range[0], iters_range[1] + 1))))
    return out


def serve_request_volume(spec: ServeRequestSpec, k: int) -> np.ndarray:
    """The halo-padded image of one request, from the generator of its source."""
    shp = spec.padded_zyx
    if spec.source == "lightsheet":
        return lightsheet_volume_u16(shp, workload=5, brick=k)
    if spec.source == "microct":
        f = MicroCTField(extent_xyz=(max(shp[2] + 64, 512), max(shp[1] + 64, 512), max(shp[0] + 64, 512)),
                         workload=500 + k)
        bs = BrickSpec((spec.halo + 8, spec.halo + 8, spec.halo + 8), tuple(reversed(spec.core_zyx)), spec.halo)
        return f.brick(bs, k)
    return milling_volume_u8(shp, workload=5, brick=k)
