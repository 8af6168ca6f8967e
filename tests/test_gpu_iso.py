"""rsf_isosurface (marching tetrahedra) against the oracle: the same keys, the
same three vertices per key within FP32 rounding, the same orientation on
non-degenerate triangles; a ball's surface is closed and outward; counting
without a buffer; host and device inputs."""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    yield c
    c.close()


def _compare(tri, keys, phi, iso=0.0):
    rk, rt = oracle.isosurface(phi.astype(np.float64), iso)
    o, ro = np.argsort(keys), np.argsort(rk)
    tri, keys, rt, rk = tri[o].astype(np.float64), keys[o], rt[ro], rk[ro]
    np.testing.assert_array_equal(keys, rk)
    # the same three points per triangle (FP32 interpolation), matched as sets
    d = np.abs(tri[:, :, None, :] - rt[:, None, :, :]).max(axis=3)
    assert np.all(d.min(axis=2).max(axis=1) < 4e-6 * max(phi.shape)), "vertex positions"
    # and the same orientation where the triangle is not degenerate
    n1 = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    n2 = np.cross(rt[:, 1] - rt[:, 0], rt[:, 2] - rt[:, 0])
    big = np.linalg.norm(n2, axis=1) > 1e-3
    assert np.all(np.einsum("ij,ij->i", n1[big], n2[big]) > 0)
    return len(keys)


def test_matches_oracle_on_a_segmentation(ctx):
    vol = synth.tree_volume_u8((20, 24, 28), n_segments=8)
    phi = ctx.evolve(torch.from_numpy(vol).cuda(), torch.from_numpy(synth.box_phi0(vol.shape, 10)).cuda(),
                     synth.RSFParams().as_dict(), 3)
    tri, keys = ctx.isosurface(phi)
    assert _compare(tri, keys, phi.cpu().numpy()) > 100


def test_ball_and_levels(ctx):
    n = 22
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    phi = (6.3 - np.sqrt((x - 10.4) ** 2 + (y - 10.7) ** 2 + (z - 10.2) ** 2)).astype(np.float32)
    for iso in (0.0, 1.25, -2.5):
        tri, keys = ctx.isosurface(torch.from_numpy(phi).cuda(), iso)
        _compare(tri, keys, phi, iso)
    tri, _ = ctx.isosurface(phi, 0.0)   # host input
    c = np.array([10.4, 10.7, 10.2])
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]).astype(np.float64)
    big = np.linalg.norm(nrm, axis=1) > 1e-3      # FP32 normals of near-degenerate triangles carry no sign
    assert big.mean() > 0.9
    assert np.all(np.einsum("ij,ij->i", nrm[big], tri.mean(axis=1)[big] - c) > 0)


def test_count_only_and_flat(ctx):
    phi = torch.full((5, 6, 7), -1.0, device="cuda")
    tri, keys = ctx.isosurface(phi)
    assert len(tri) == 0 and len(keys) == 0
