"""Pins of the oracle's volume-level curtain scheme (Sec. 4.1): sub-volumes
evolved independently, merged by linear interpolation across the curtain.

* One sub-volume (edge >= every dimension) is the plain evolution, bit for bit.
* Zero iterations give phi0 back (the weights are a normalised partition).
* Across an overlap of exactly the curtain width the two weights sum to one:
  the merge is the linear interpolation between the neighbours.
* The merge is a convex combination of the sub-volume results.
* Away from the seams the scheme is the whole-volume evolution, bit for bit:
  after n iterations a voxel depends only on voxels within n * 2R (the fits'
  convolution of a convolution), so a voxel that only one sub-volume covers,
  farther than that from the sub-volume's interior faces, is unaffected by
  the split.
"""
import numpy as np

import oracle
from paper_2404_02813_gb300 import synth

P = dict(sigma=1.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)


def _case(shape=(30, 34, 40)):
    vol = synth.tree_volume_u8(shape, n_segments=12).astype(np.float64)
    phi0 = synth.mean_rule_phi0(vol.astype(np.uint8)).astype(np.float64)
    return vol, phi0


def test_starts_cover_with_overlap():
    for n, edge, c in [(100, 40, 10), (95, 40, 10), (41, 40, 10), (30, 40, 10), (64, 24, 4)]:
        s = oracle.curtain_starts(n, edge, c)
        ends = [min(a + edge, n) for a in s]
        assert s[0] == 0 and ends[-1] == n
        for a, b in zip(ends[:-1], s[1:]):
            assert a - b >= min(c, edge)  # neighbours overlap by at least the curtain


def test_linear_interpolation_across_a_curtain_wide_overlap():
    n, c = 70, 10
    x = np.arange(30, 40, dtype=np.float64)
    h0 = oracle.curtain_weight(x, 0, 40, n, c)
    h1 = oracle.curtain_weight(x, 30, 70, n, c)
    np.testing.assert_allclose(h0 + h1, 1.0, rtol=0, atol=1e-15)
    assert np.all(np.diff(h1) > 0) and np.all(np.diff(h0) < 0)
    np.testing.assert_allclose(np.diff(h1), 1.0 / c, rtol=1e-12)


def test_single_subvolume_is_plain_evolution():
    vol, phi0 = _case()
    a = oracle.curtain_evolve(vol, phi0, P, 3, edge=64, curtain=4)
    b = oracle.evolve(vol, phi0, P, 3)
    np.testing.assert_array_equal(a, b)


def test_zero_iterations_return_phi0():
    vol, phi0 = _case()
    a = oracle.curtain_evolve(vol, phi0, P, 0, edge=16, curtain=4)
    np.testing.assert_allclose(a, phi0, rtol=1e-15, atol=0)


def test_merge_is_a_convex_combination():
    vol, phi0 = _case()
    edge, c, it = 20, 5, 2
    merged = oracle.curtain_evolve(vol, phi0, P, it, edge=edge, curtain=c)
    lo = np.full(vol.shape, np.inf)
    hi = np.full(vol.shape, -np.inf)
    nz, ny, nx = vol.shape
    for z0 in oracle.curtain_starts(nz, edge, c):
        for y0 in oracle.curtain_starts(ny, edge, c):
            for x0 in oracle.curtain_starts(nx, edge, c):
                sl = np.s_[z0:z0 + edge, y0:y0 + edge, x0:x0 + edge]
                sub = oracle.evolve(vol[sl], phi0[sl], P, it)
                lo[sl] = np.minimum(lo[sl], sub)
                hi[sl] = np.maximum(hi[sl], sub)
    tol = 1e-12 * np.maximum(1.0, np.abs(merged))
    assert np.all(merged >= lo - tol) and np.all(merged <= hi + tol)


def test_equals_whole_volume_away_from_the_seams():
    vol, phi0 = _case((34, 36, 60))
    edge, c, it = 32, 4, 2
    R = 2                                   # round(2 * sigma) for sigma = 1
    reach = it * 2 * R
    merged = oracle.curtain_evolve(vol, phi0, P, it, edge=edge, curtain=c)
    whole = oracle.evolve(vol, phi0, P, it)
    nz, ny, nx = vol.shape
    count = np.zeros(vol.shape, dtype=int)
    safe = np.zeros(vol.shape, dtype=bool)
    for z0 in oracle.curtain_starts(nz, edge, c):
        for y0 in oracle.curtain_starts(ny, edge, c):
            for x0 in oracle.curtain_starts(nx, edge, c):
                box = [(z0, min(z0 + edge, nz), nz), (y0, min(y0 + edge, ny), ny), (x0, min(x0 + edge, nx), nx)]
                sl = tuple(slice(s, e) for s, e, _ in box)
                count[sl] += 1
                ok = np.ones(vol.shape, dtype=bool)
                for ax, (s, e, n) in enumerate(box):
                    idx = np.arange(n)
                    far = (idx >= s) & (idx < e)
                    if s > 0:
                        far &= idx >= s + reach
                    if e < n:
                        far &= idx < e - reach
                    shape = [1, 1, 1]
                    shape[ax] = n
                    ok &= far.reshape(shape)
                safe |= ok
    sel = safe & (count == 1)
    assert sel.sum() > 1000
    np.testing.assert_array_equal(merged[sel], whole[sel])
    # and the seams do differ somewhere (the split is not a no-op)
    assert np.abs(merged - whole).max() > 0
