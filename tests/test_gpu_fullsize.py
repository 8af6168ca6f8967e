"""Parity at the benchmark's full size and launch configuration: the 512^3
uint16 light-sheet workload at sigma = 3 on the default schedule (tiled, FP32
storage, default z chunk), one iteration from the state after two, checked on
sampled voxels against the oracle's direct-sum evaluation of the update at a
single voxel (Eqs. 1, 6-14 with triple sums, no separable passes).

Samples: the eight corners, face and edge voxels, the boundaries of the x/y
tiles (multiples of 32 in x, of 8 and 32 in y), of the z chunks and slabs
(multiples of 64 and 8 in z), and random interior voxels.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import phi_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E = 512
P_LIGHTSHEET = 4300.0


def _samples(rng):
    pts = set()
    ends = (0, E - 1)
    for x in ends:
        for y in ends:
            for z in ends:
                pts.add((x, y, z))
    tile_x = (0, 1, 31, 32, 33, 255, 256, 480, 510, 511)
    tile_y = (0, 1, 7, 8, 31, 32, 263, 264, 504, 511)
    tile_z = (0, 1, 7, 8, 63, 64, 65, 127, 128, 447, 448, 510, 511)
    for _ in range(60):
        pts.add((int(rng.choice(tile_x)), int(rng.choice(tile_y)), int(rng.choice(tile_z))))
    while len(pts) < 128:
        pts.add(tuple(int(v) for v in rng.integers(0, E, size=3)))
    return sorted(pts)


def test_fullsize_lightsheet_sampled_voxels():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol = synth.lightsheet_volume_u16((E, E, E), brick=0)
    phi0 = synth.mean_rule_phi0(vol)
    p = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P_LIGHTSHEET ** 2, mu=1.0, dt=0.1)
    ctx = rsf.Context(0)
    try:
        v = torch.from_numpy(vol).cuda()
        phi_n = ctx.evolve(v, torch.from_numpy(phi0).cuda(), p, 2)
        nxt = ctx.evolve(v, phi_n, p, 1).cpu().numpy()
        phi_n = phi_n.cpu().numpy()
    finally:
        ctx.close()
    I64 = np.ascontiguousarray(vol, dtype=np.float64)
    P64 = np.ascontiguousarray(phi_n, dtype=np.float64)
    pts = _samples(np.random.default_rng(2404))
    worst = 0.0
    for (x, y, z) in pts:
        ref = oracle.point_next(I64, P64, p, x, y, z)
        got = float(nxt[z, y, x])
        tol = float(phi_tol(np.array([P64[z, y, x]]), np.array([ref]))[0])
        assert np.isfinite(got), f"non-finite phi at {(x, y, z)}"
        assert abs(got - ref) <= tol, f"voxel {(x, y, z)}: gpu {got!r} oracle {ref!r} tol {tol:.3e}"
        worst = max(worst, abs(got - ref) / tol)
    print(f"{len(pts)} sampled voxels, worst |d|/tol = {worst:.3f}")


def test_fullsize_paper500_eq15_sampled_voxels():
    """The paper's Table 1 configuration as the benchmark runs it: 500^3 uint8
    milling-like volume, Eq. (15) with sigma_2 = 0, the 3-D parameters of Sec. 5.3
    (sigma_1 = 5, dt = 0.06, alpha = 255^2 * 0.0009, beta = 0.1), FP32 storage."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    e = 500
    vol = synth.field_volume(synth.MillingField(extent_xyz=(e, e, e), workload=6))
    phi0 = synth.mean_rule_phi0(vol)
    p = dict(sigma=5.0, eps=1.0, lambda1=0.1, lambda2=0.1, nu=255.0 * 255.0 * 0.0009, mu=1.0, dt=0.06)
    ctx = rsf.Context(0)
    try:
        ctx.set_force("eq15")
        v = torch.from_numpy(vol).cuda()
        phi_n = ctx.evolve(v, torch.from_numpy(phi0).cuda(), p, 2)
        nxt = ctx.evolve(v, phi_n, p, 1).cpu().numpy()
        phi_n = phi_n.cpu().numpy()
    finally:
        ctx.close()
    I64 = vol.astype(np.float64)
    P64 = phi_n.astype(np.float64)
    rng = np.random.default_rng(500)
    pts = {(x, y, z) for x in (0, e - 1) for y in (0, e - 1) for z in (0, e - 1)}
    edges = (0, 1, 31, 32, 255, 256, 479, 480, 498, 499)
    for _ in range(40):
        pts.add(tuple(int(rng.choice(edges)) for _ in range(3)))
    while len(pts) < 96:
        pts.add(tuple(int(v) for v in rng.integers(0, e, size=3)))
    worst = 0.0
    for (x, y, z) in sorted(pts):
        ref = oracle.point_next(I64, P64, p, x, y, z, force="eq15")
        got = float(nxt[z, y, x])
        tol = float(phi_tol(np.array([P64[z, y, x]]), np.array([ref]))[0])
        assert abs(got - ref) <= tol, f"voxel {(x, y, z)}: gpu {got!r} oracle {ref!r} tol {tol:.3e}"
        worst = max(worst, abs(got - ref) / tol)
    print(f"paper500 eq15: {len(pts)} sampled voxels, worst |d|/tol = {worst:.3f}")
