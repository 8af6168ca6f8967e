"""Pins of the oracle's seed initialisation (Sec. 4.3): determinant-of-Hessian
blob seeds per z slice and phi0 = r0 - distance to the nearest seed.

* The Hessian filters equal scipy's Gaussian derivative filters (same sampled
  kernels, zero padding, one z slice at a time).
* A Gaussian blob gives one seed, at its centre, in every slice; of two blobs
  the threshold keeps both or only the stronger.
* phi0 equals r0 minus scipy's exact Euclidean distance transform, and for a
  single seed r0 minus the closed-form distance.
"""
import numpy as np
import pytest

import oracle

ndi = pytest.importorskip("scipy.ndimage")


def _blobs(n=40, nz=3, centres=((12.0, 14.0, 170.0), (28.0, 26.0, 60.0)), w=2.5):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(n), np.arange(n), indexing="ij")
    I = np.full((nz, n, n), 30.0)
    for cy, cx, a in centres:
        I += a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))
    return I


@pytest.mark.parametrize("s", [1.0, 1.7, 2.5])
def test_hessian_filters_match_scipy(s):
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 255, size=(4, 23, 29))
    D = oracle.doh_response(I, s)
    kw = dict(sigma=(0.0, s, s), mode="constant", cval=0.0, truncate=3.0)
    Ixx = ndi.gaussian_filter(I, order=(0, 0, 2), **kw)
    Iyy = ndi.gaussian_filter(I, order=(0, 2, 0), **kw)
    Ixy = ndi.gaussian_filter(I, order=(0, 1, 1), **kw)
    ref = np.where(Ixx + Iyy < 0, s ** 4 * (Ixx * Iyy - Ixy * Ixy), -np.inf)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(D))
    np.testing.assert_allclose(D[fin], ref[fin], rtol=1e-10, atol=1e-9 * np.abs(ref[fin]).max())


def test_blob_centre_is_the_seed():
    I = _blobs(centres=((17.0, 21.0, 170.0),))
    seeds = np.argwhere(oracle.doh_seeds(I, 2.0, 0.1))
    assert seeds.tolist() == [[0, 17, 21], [1, 17, 21], [2, 17, 21]]


def test_threshold_selects_by_strength():
    I = _blobs()
    both = {tuple(p[1:]) for p in np.argwhere(oracle.doh_seeds(I, 2.0, 0.05))}
    strong = {tuple(p[1:]) for p in np.argwhere(oracle.doh_seeds(I, 2.0, 0.5))}
    assert both == {(12, 14), (28, 26)}
    assert strong == {(12, 14)}


def test_phi0_is_r0_minus_euclidean_distance():
    rng = np.random.default_rng(9)
    shape = (9, 11, 13)
    mask = rng.random(shape) < 0.02
    mask[4, 5, 6] = True
    phi = oracle.seed_phi0(shape, np.argwhere(mask), 2.0)
    d = ndi.distance_transform_edt(~mask)
    np.testing.assert_allclose(phi, 2.0 - d, rtol=0, atol=1e-12)


def test_single_seed_closed_form():
    phi = oracle.seed_phi0((6, 7, 8), np.array([[2, 3, 4]]), 1.5)
    for (z, y, x) in [(0, 0, 0), (2, 3, 4), (5, 6, 7), (2, 0, 4)]:
        assert abs(phi[z, y, x] - (1.5 - np.sqrt((z - 2) ** 2 + (y - 3) ** 2 + (x - 4) ** 2))) < 1e-14
