"""FP64 CPU oracle of the 3D RSF level-set iteration (arXiv 2404.02813).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product path (``paper_2404_02813_gb300``) never imports it, and the two
share no code: the C source ``rsf_oracle.c`` restates every equation on its
own.

Functions follow the paper's equations (see the header of ``rsf_oracle.c``
for the full list and for the readings taken where the paper is silent):

* :func:`taps`        Eq. (7): normalised discrete Gaussian, R = round(2 sigma)
* :func:`conv3`       Eq. (6) convolution K*F, separable x -> y -> z, zero padding
* :func:`heaviside`   Eq. (10)
* :func:`dirac`       Eq. (14)
* :func:`stencils`    Eqs. (3)-(4): curvature div(grad phi/|grad phi|), Laplacian
* :func:`step`        one iteration, Eqs. (1), (6), (11)-(14)
* :func:`evolve`      ``iters`` iterations
* :func:`point_next`  one voxel of :func:`step` by direct triple sums
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsf_oracle.c")
_LIBS = {False: os.path.join(_HERE, "liboracle.so"), True: os.path.join(_HERE, "liboracle_omp.so")}

DUMP_NAMES = ("H", "f1", "f2", "e1", "e2", "g", "kappa", "lap")


def build(force: bool = False) -> None:
    """Compile the single-thread and the OpenMP builds of the oracle with gcc.

    Both use -O2 without fast-math, so IEEE double arithmetic is kept.
    """
    for omp, out in _LIBS.items():
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
               _SRC, "-o", out + ".tmp", "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


_loaded = {}


def _lib(omp: bool = False):
    if omp in _loaded:
        return _loaded[omp]
    build()
    lib = ctypes.CDLL(_LIBS[omp])
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    d = ctypes.c_double
    lib.rsf_oracle_radius.argtypes = [d]
    lib.rsf_oracle_radius.restype = ctypes.c_int
    lib.rsf_oracle_taps.argtypes = [d, dp]
    lib.rsf_oracle_taps.restype = ctypes.c_int
    lib.rsf_oracle_conv3.argtypes = [dp, dp, i64, i64, i64, d]
    lib.rsf_oracle_conv3.restype = None
    lib.rsf_oracle_heaviside.argtypes = [d, d]
    lib.rsf_oracle_heaviside.restype = d
    lib.rsf_oracle_dirac.argtypes = [d, d]
    lib.rsf_oracle_dirac.restype = d
    lib.rsf_oracle_stencils.argtypes = [dp, i64, i64, i64, dp, dp]
    lib.rsf_oracle_stencils.restype = None
    lib.rsf_oracle_step.argtypes = [dp, dp, dp, i64, i64, i64, d, d, d, d, d, d, d, dp, ctypes.c_int]
    lib.rsf_oracle_step.restype = None
    lib.rsf_oracle_evolve.argtypes = [dp, dp, dp, i64, i64, i64, d, d, d, d, d, d, d, ctypes.c_int, ctypes.c_int]
    lib.rsf_oracle_evolve.restype = None
    lib.rsf_oracle_point_next.argtypes = [dp, dp, i64, i64, i64, i64, i64, i64, d, d, d, d, d, d, d, dp,
                                          ctypes.c_int]
    lib.rsf_oracle_point_next.restype = d
    lib.rsf_oracle_dump_slots.argtypes = []
    lib.rsf_oracle_dump_slots.restype = ctypes.c_int
    _loaded[omp] = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vol(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 3:
        raise ValueError("expected a 3-D [nz, ny, nx] array")
    return a


def radius(sigma: float) -> int:
    return int(_lib().rsf_oracle_radius(float(sigma)))


def taps(sigma: float) -> np.ndarray:
    R = radius(sigma)
    g = np.zeros(2 * R + 1, dtype=np.float64)
    _lib().rsf_oracle_taps(float(sigma), _dp(g))
    return g


def conv3(F, sigma: float, omp: bool = False) -> np.ndarray:
    F = _vol(F)
    nz, ny, nx = F.shape
    out = np.empty_like(F)
    _lib(omp).rsf_oracle_conv3(_dp(F), _dp(out), nx, ny, nz, float(sigma))
    return out


def heaviside(u, eps: float = 1.0) -> np.ndarray:
    f = _lib().rsf_oracle_heaviside
    u = np.asarray(u, dtype=np.float64)
    return np.vectorize(lambda v: f(float(v), float(eps)), otypes=[np.float64])(u)


def dirac(u, eps: float = 1.0) -> np.ndarray:
    f = _lib().rsf_oracle_dirac
    u = np.asarray(u, dtype=np.float64)
    return np.vectorize(lambda v: f(float(v), float(eps)), otypes=[np.float64])(u)


def stencils(phi, omp: bool = False):
    """Return (kappa, laplacian) of ``phi``."""
    phi = _vol(phi)
    nz, ny, nx = phi.shape
    kap = np.empty_like(phi)
    lap = np.empty_like(phi)
    _lib(omp).rsf_oracle_stencils(_dp(phi), nx, ny, nz, _dp(kap), _dp(lap))
    return kap, lap


def _params(p: dict):
    return (float(p["sigma"]), float(p["eps"]), float(p["lambda1"]), float(p["lambda2"]),
            float(p["nu"]), float(p["mu"]), float(p["dt"]))


# Data-term forms: "li" (Li et al.'s e_i with K*1 and K*f_i, Eqs. 11-12 as read)
# and "eq15" (the paper's Eq. 15 with sigma_2 = 0: e_i = (I - f_i)^2).
FORCES = {"li": 0, "eq15": 1}


def _force(force: str) -> int:
    if force not in FORCES:
        raise ValueError(f"unknown force form {force!r}; expected one of {sorted(FORCES)}")
    return FORCES[force]


def step(I, phi, params: dict, dump: bool = False, omp: bool = False, force: str = "li"):
    """One iteration. Returns phi_next, or (phi_next, {stage: array}) with ``dump``."""
    I = _vol(I)
    phi = _vol(phi)
    if I.shape != phi.shape:
        raise ValueError("I and phi shapes differ")
    nz, ny, nx = I.shape
    out = np.empty_like(phi)
    lib = _lib(omp)
    nslots = lib.rsf_oracle_dump_slots()
    buf: Optional[np.ndarray] = np.empty((nslots,) + I.shape, dtype=np.float64) if dump else None
    lib.rsf_oracle_step(_dp(I), _dp(phi), _dp(out), nx, ny, nz, *_params(params),
                        _dp(buf) if dump else None, _force(force))
    if dump:
        return out, {name: buf[i] for i, name in enumerate(DUMP_NAMES)}
    return out


def evolve(I, phi0, params: dict, iters: int, omp: bool = False, force: str = "li") -> np.ndarray:
    I = _vol(I)
    phi0 = _vol(phi0)
    if I.shape != phi0.shape:
        raise ValueError("I and phi0 shapes differ")
    nz, ny, nx = I.shape
    out = np.empty_like(phi0)
    _lib(omp).rsf_oracle_evolve(_dp(I), _dp(phi0), _dp(out), nx, ny, nz, *_params(params), int(iters),
                                _force(force))
    return out


POINT_TERMS = ("e1", "e2", "g", "kappa", "lap")


def point_next(I, phi, params: dict, x: int, y: int, z: int, terms: bool = False, force: str = "li"):
    """phi_{n+1} at voxel (x, y, z) by direct triple sums (no separable passes).

    With ``terms``, returns (phi_next, {e1, e2, g, kappa, lap}) at the voxel."""
    I = _vol(I)
    phi = _vol(phi)
    nz, ny, nx = I.shape
    t = np.zeros(len(POINT_TERMS), dtype=np.float64)
    v = float(_lib().rsf_oracle_point_next(_dp(I), _dp(phi), nx, ny, nz, int(x), int(y), int(z),
                                           *_params(params), _dp(t) if terms else None, _force(force)))
    return (v, dict(zip(POINT_TERMS, t.tolist()))) if terms else v


# ------------------------------------------------ volume-level curtain scheme
#
# Sec. 4.1: a large volume is divided into sub-volumes processed independently,
# overlapping by a curtain region, and neighbouring results are merged by linear
# interpolation across the curtain.  Reading (the paper gives no formula):
#   * along each axis of length n, sub-volumes of `edge` voxels start at
#     multiples of edge - curtain; the last one is moved to end at n (one
#     sub-volume when edge >= n); neighbours overlap by at least `curtain`;
#   * sub-volume b has the weight w_b(x) = prod over axes of h_b(x_a), with
#     h = 1 inside, rising linearly over the `curtain` voxels after each face
#     interior to the volume: h = min(1, (x - s + 1/2)/curtain) after a start
#     face s > 0 and min(1, (e - x - 1/2)/curtain) before an end face e < n;
#   * the merged phi is sum_b w_b phi_b / sum_b w_b, which is the linear
#     interpolation across an overlap of exactly `curtain` voxels.
# Every sub-volume is evolved as its own volume (its own zero padding and
# reflect-101 faces).

def curtain_starts(n: int, edge: int, curtain: int) -> list:
    if edge >= n:
        return [0]
    step = edge - curtain
    starts = list(range(0, n - edge, step))
    return starts + [n - edge]


def curtain_weight(x: np.ndarray, s: int, e: int, n: int, curtain: int) -> np.ndarray:
    h = np.ones(x.shape, dtype=np.float64)
    if s > 0:
        h = np.minimum(h, (x - s + 0.5) / curtain)
    if e < n:
        h = np.minimum(h, (e - x - 0.5) / curtain)
    return np.clip(h, 0.0, 1.0)


def curtain_evolve(I, phi0, params: dict, iters: int, edge: int, curtain: int, omp: bool = False,
                   force: str = "li") -> np.ndarray:
    """The curtain scheme: every sub-volume evolved by `evolve`, then merged."""
    I = _vol(I)
    phi0 = _vol(phi0)
    nz, ny, nx = I.shape
    num = np.zeros(I.shape, dtype=np.float64)
    den = np.zeros(I.shape, dtype=np.float64)
    for z0 in curtain_starts(nz, edge, curtain):
        z1 = min(z0 + edge, nz)
        wz = curtain_weight(np.arange(z0, z1, dtype=np.float64), z0, z1, nz, curtain)
        for y0 in curtain_starts(ny, edge, curtain):
            y1 = min(y0 + edge, ny)
            wy = curtain_weight(np.arange(y0, y1, dtype=np.float64), y0, y1, ny, curtain)
            for x0 in curtain_starts(nx, edge, curtain):
                x1 = min(x0 + edge, nx)
                wx = curtain_weight(np.arange(x0, x1, dtype=np.float64), x0, x1, nx, curtain)
                sub = evolve(I[z0:z1, y0:y1, x0:x1], phi0[z0:z1, y0:y1, x0:x1], params, iters, omp=omp,
                             force=force)
                w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                num[z0:z1, y0:y1, x0:x1] += w * sub
                den[z0:z1, y0:y1, x0:x1] += w
    return num / den


# ---------------------------------------------------- initialisation (Sec. 4.3)
#
# Seeds: per z slice, determinant-of-Hessian blob detection.  Reading (the paper
# names the detector, not its discretisation):
#   * taps of the sampled Gaussian and of its first and second derivatives,
#     k = -R..R with R = round(3 sigma): g_k = exp(-k^2/2s^2) / sum_j exp(-j^2/2s^2),
#     g'_k = -(k/s^2) g_k, g''_k = (k^2/s^4 - 1/s^2) g_k;
#   * in-slice filtering by correlation with zero padding:
#     I_xx = (g'' along x, g along y), I_yy = (g along x, g'' along y),
#     I_xy = (g' along x, g' along y);
#   * D = s^4 (I_xx I_yy - I_xy^2) (scale-normalised), kept where
#     I_xx + I_yy < 0 (bright blobs), else -inf;
#   * a voxel is a seed when D > t * max of D over its slice (t the relative
#     threshold, the maximum positive) and D exceeds D at each of its in-slice
#     neighbours (the 8 that exist).
# phi0 = r0 - d, d the Euclidean distance to the nearest seed (the distance
# the paper's fast sweeping approximates; here exact).

def deriv_taps(s: float):
    R = int(np.floor(3.0 * s + 0.5))
    k = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * s * s))
    g /= g.sum()
    return k, g, -(k / (s * s)) * g, (k * k / s ** 4 - 1.0 / (s * s)) * g


def _corr_axis(F: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    """out(i) = sum_k w_k F(i + k) along `axis`, zero outside."""
    R = (w.size - 1) // 2
    pad = [(0, 0)] * F.ndim
    pad[axis] = (R, R)
    P = np.pad(F, pad)
    out = np.zeros_like(F)
    n = F.shape[axis]
    for j in range(w.size):
        sl = [slice(None)] * F.ndim
        sl[axis] = slice(j, j + n)
        out += w[j] * P[tuple(sl)]
    return out


def doh_response(I, s: float) -> np.ndarray:
    """D per voxel ([z, y, x]; each z slice filtered on its own)."""
    I = _vol(I)
    _, g, g1, g2 = deriv_taps(s)
    Ixx = _corr_axis(_corr_axis(I, g2, 2), g, 1)
    Iyy = _corr_axis(_corr_axis(I, g, 2), g2, 1)
    Ixy = _corr_axis(_corr_axis(I, g1, 2), g1, 1)
    D = s ** 4 * (Ixx * Iyy - Ixy * Ixy)
    return np.where(Ixx + Iyy < 0.0, D, -np.inf)


def doh_seeds(I, s: float, rel_threshold: float) -> np.ndarray:
    """Boolean seed mask."""
    return seeds_from_response(doh_response(I, s), rel_threshold)


def seeds_from_response(D: np.ndarray, rel_threshold: float) -> np.ndarray:
    """The seed rule applied to a response field D ([z, y, x])."""
    nz, ny, nx = D.shape
    smax = D.reshape(nz, -1).max(axis=1)
    seeds = (D > rel_threshold * smax[:, None, None]) & (smax[:, None, None] > 0.0)
    P = np.pad(D, ((0, 0), (1, 1), (1, 1)), constant_values=-np.inf)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            seeds &= D > P[:, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return seeds


def seed_phi0(shape, seeds_zyx: np.ndarray, r0: float) -> np.ndarray:
    """phi0 = r0 - (Euclidean distance to the nearest seed), by brute force."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    best = np.full(shape, np.inf)
    for sz, sy, sx in np.asarray(seeds_zyx, dtype=np.int64):
        best = np.minimum(best, (z - sz) ** 2 + (y - sy) ** 2 + (x - sx) ** 2)
    return r0 - np.sqrt(best)


# ------------------------------------------------------- validation (Sec. 5.3)
# The paper scores segmentations by the Dice coefficient and the Jaccard index
# against annotations; here against the synthetic generators' ground truth.

def overlap_counts(phi, truth) -> tuple:
    """(|phi > 0|, |truth|, |phi > 0 and truth|)."""
    seg = np.asarray(phi) > 0
    t = np.asarray(truth).astype(bool)
    return int(seg.sum()), int(t.sum()), int(np.logical_and(seg, t).sum())


def dice_jaccard(counts) -> tuple:
    a, b, c = counts
    return (2.0 * c / (a + b) if a + b else 1.0), (c / (a + b - c) if a + b - c else 1.0)


# ------------------------------------------------- isosurface (Figs. 8-9)
#
# The zero level set as triangles, by marching tetrahedra: every voxel cube
# (x..x+1, y..y+1, z..z+1) is split into six tetrahedra along its main
# diagonal, one per order of the axes: corners 0, e_a, e_a + e_b, (1,1,1) for
# the permutation (a, b, c).  In a tetrahedron with k corners where phi > iso:
# k = 0 or 4, no triangle; k = 1 or 3, one triangle on the three edges that
# join the odd corner to the others; k = 2, two triangles on the four crossed
# edges (the quadrilateral p0 p1 q1 q0 split along p0-q1, in the order the
# edges are listed below).  An edge (p, q), p the corner of smaller grid index,
# is crossed at p + t (q - p), t = (iso - phi_p) / (phi_q - phi_p).  Each triangle is keyed by
# (cube index) * 12 + (tetrahedron) * 2 + (triangle within it), the cube index
# (z * (ny-1) + y) * (nx-1) + x, so that sets of triangles compare by key.
# A grid value equal to iso counts as outside; the crossings of its edges then
# meet at that corner and the triangles around it are degenerate.
# Orientation: the normal (v1 - v0) x (v2 - v0) points from phi > iso towards
# phi < iso (from the odd corner for k = 1, towards it for k = 3, from the
# inside edge's midpoint to the outside edge's for k = 2); otherwise v1 and v2
# are swapped.

TETRA_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _tetra_corners(perm):
    c0 = (0, 0, 0)
    c1 = [0, 0, 0]
    c1[perm[0]] = 1
    c2 = list(c1)
    c2[perm[1]] = 1
    return [c0, tuple(c1), tuple(c2), (1, 1, 1)]


def isosurface(phi, iso: float = 0.0):
    """(keys [T], triangles [T, 3, 3] as (x, y, z) points) of the phi = iso surface."""
    phi = _vol(phi)
    nz, ny, nx = phi.shape
    keys, tris = [], []
    for z in range(nz - 1):
        for y in range(ny - 1):
            for x in range(nx - 1):
                base = ((z * (ny - 1) + y) * (nx - 1) + x) * 12
                for t, perm in enumerate(TETRA_PERMS):
                    cs = _tetra_corners(perm)
                    pts = [np.array([x + c[0], y + c[1], z + c[2]], dtype=np.float64) for c in cs]
                    val = [phi[z + c[2], y + c[1], x + c[0]] for c in cs]
                    ins = [v > iso for v in val]
                    k = sum(ins)
                    if k in (0, 4):
                        continue

                    def cut(i, j):
                        # from the corner with the smaller grid index, so that an edge
                        # shared by several tetrahedra gives the same point in each
                        if (cs[i][2], cs[i][1], cs[i][0]) > (cs[j][2], cs[j][1], cs[j][0]):
                            i, j = j, i
                        s = (iso - val[i]) / (val[j] - val[i])
                        return pts[i] + s * (pts[j] - pts[i])

                    def oriented(tri, out_dir):
                        # normal (v1 - v0) x (v2 - v0) towards phi < iso
                        nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
                        return [tri[0], tri[2], tri[1]] if np.dot(nrm, out_dir) < 0 else tri

                    if k in (1, 3):
                        odd = ins.index(k == 1)
                        others = [i for i in range(4) if i != odd]
                        tri = [cut(odd, others[0]), cut(odd, others[1]), cut(odd, others[2])]
                        out_dir = (tri[0] - pts[odd]) if k == 1 else (pts[odd] - tri[0])
                        keys.append(base + 2 * t)
                        tris.append(oriented(tri, out_dir))
                    else:
                        a = [i for i in range(4) if ins[i]]
                        b = [i for i in range(4) if not ins[i]]
                        p0, p1 = cut(a[0], b[0]), cut(a[0], b[1])
                        q0, q1 = cut(a[1], b[0]), cut(a[1], b[1])
                        out_dir = (pts[b[0]] + pts[b[1]] - pts[a[0]] - pts[a[1]]) / 2.0
                        keys.append(base + 2 * t)
                        tris.append(oriented([p0, p1, q1], out_dir))
                        keys.append(base + 2 * t + 1)
                        tris.append(oriented([p0, q1, q0], out_dir))
    return np.array(keys, dtype=np.int64), np.array(tris, dtype=np.float64).reshape(-1, 3, 3)
