"""Pins of the oracle's segmentation scores (Dice, Jaccard; Sec. 5.3): two
axis-aligned boxes with a known intersection, the identity Dice = 2J/(1+J),
and the identical and disjoint cases."""
import numpy as np

import oracle


def _box(shape, lo, hi):
    m = np.zeros(shape, dtype=bool)
    m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = True
    return m


def test_two_boxes():
    shape = (20, 22, 24)
    a = _box(shape, (2, 3, 4), (12, 13, 14))        # 10^3 = 1000 voxels
    b = _box(shape, (7, 8, 9), (17, 18, 19))        # 1000 voxels, overlap 5^3 = 125
    phi = np.where(a, 1.5, -1.5)
    counts = oracle.overlap_counts(phi, b)
    assert counts == (1000, 1000, 125)
    d, j = oracle.dice_jaccard(counts)
    assert abs(d - 250.0 / 2000.0) < 1e-15 and abs(j - 125.0 / 1875.0) < 1e-15
    assert abs(d - 2 * j / (1 + j)) < 1e-15


def test_identical_and_disjoint():
    shape = (8, 8, 8)
    a = _box(shape, (1, 1, 1), (4, 5, 6))
    assert oracle.dice_jaccard(oracle.overlap_counts(np.where(a, 1.0, -1.0), a)) == (1.0, 1.0)
    b = _box(shape, (5, 5, 6), (8, 8, 8))
    assert oracle.dice_jaccard(oracle.overlap_counts(np.where(a, 1.0, -1.0), b)) == (0.0, 0.0)
    # phi = 0 is outside (the segmentation is phi > 0)
    assert oracle.overlap_counts(np.zeros(shape), a)[0] == 0
