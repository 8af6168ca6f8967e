"""Pins of the oracle's isosurface of phi = iso (marching tetrahedra).

* A plane phi = z - h: every vertex lies on z = h and the area is the box's
  cross-section (linear interpolation is exact for a linear phi).
* A ball (phi > 0 inside): a closed surface, every edge shared by two
  triangles, Euler characteristic 2, normals pointing away from the centre,
  vertices within a fraction of a voxel of the radius, area within 2 % of 4 pi r^2.
* Two disjoint balls: Euler characteristic 4.
"""
import numpy as np

import oracle


def _area(T):
    return 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1).sum()


def _euler(T):
    _, inv = np.unique(T.reshape(-1, 3), axis=0, return_inverse=True)  # shared edges give identical points
    tri = inv.reshape(-1, 3)
    edges = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    ue, cnt = np.unique(edges, axis=0, return_counts=True)
    return int(inv.max() + 1) - len(ue) + len(tri), cnt


def _ball_phi(n, centres, r):
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    d = np.full((n, n, n), np.inf)
    for c in centres:
        d = np.minimum(d, np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2))
    return r - d


def test_plane():
    nz, ny, nx = 7, 9, 11
    z = np.broadcast_to(np.arange(nz, dtype=np.float64)[:, None, None], (nz, ny, nx))
    keys, T = oracle.isosurface(z - 3.3)
    assert len(keys) == len(set(keys.tolist()))
    np.testing.assert_allclose(T[..., 2], 3.3, rtol=0, atol=1e-12)
    assert abs(_area(T) - (nx - 1) * (ny - 1)) < 1e-9


def test_ball_is_closed_oriented_and_round():
    c, r = (9.5, 9.7, 9.2), 6.3
    keys, T = oracle.isosurface(_ball_phi(20, [c], r))
    chi, cnt = _euler(T)
    assert chi == 2 and np.all(cnt == 2)
    d = np.linalg.norm(T - np.array(c), axis=2)
    assert d.min() > r - 0.1 and d.max() < r + 1e-9
    n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
    assert np.all(np.einsum("ij,ij->i", n, T.mean(axis=1) - np.array(c)) > 0)
    assert abs(_area(T) / (4 * np.pi * r * r) - 1) < 0.02


def test_two_balls():
    # (a radius that puts no grid value exactly on the level: there the crossings of
    # several edges meet at the corner and the triangles around it degenerate)
    keys, T = oracle.isosurface(_ball_phi(24, [(6.2, 6.4, 6.1), (16.3, 15.8, 16.6)], 4.1234))
    chi, cnt = _euler(T)
    assert chi == 4 and np.all(cnt == 2)
