"""The seeded synthetic inputs (CPU): the generators hold none of the method's
arithmetic, but the design's input recipe rests on their properties.

* Seeds: the same (workload, brick) gives the same volume; another brick another.
* Capsule rasterisation: occupancy clip(r - d + 0.5, 0, 1) at the distance d
  to the segment, max-composited; a box of the field equals that region of a
  larger box.
* The milling field: any box equals that region of the whole (blur margin and
  per-plane noise), which is what lets 1024^3 be built slab by slab.
* The micro-CT bricks: padded shape = core + 2 halo; cores and origins in range.
* The light-sheet truth mask is occupancy >= 1/2 before the blur.
* The mean-rule phi0 built slab by slab equals the whole-volume rule.
* The serving mix: sigma from the set, halo round(3 sigma), cores in range.
"""
import numpy as np
import pytest

from paper_2404_02813_gb300 import synth

ndi = pytest.importorskip("scipy.ndimage")


def test_seeds_are_reproducible_and_distinct():
    a = synth.tree_volume_u8((24, 20, 28), brick=3, n_segments=6)
    b = synth.tree_volume_u8((24, 20, 28), brick=3, n_segments=6)
    c = synth.tree_volume_u8((24, 20, 28), brick=4, n_segments=6)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()
    assert a.dtype == np.uint8 and a.shape == (24, 20, 28)


def test_capsule_occupancy_is_clipped_distance():
    seg = synth.Segments(np.array([[4.0, 10.0, 10.0]]), np.array([[16.0, 10.0, 10.0]]), np.array([2.0]))
    occ = synth.rasterize(seg, (0, 0, 0), (20, 20, 20))
    z, y, x = np.meshgrid(np.arange(20.0), np.arange(20.0), np.arange(20.0), indexing="ij")
    t = np.clip((x - 4.0) / 12.0, 0.0, 1.0)
    d = np.sqrt((x - (4.0 + 12.0 * t)) ** 2 + (y - 10.0) ** 2 + (z - 10.0) ** 2)
    ref = np.clip(2.0 - d + 0.5, 0.0, 1.0)
    np.testing.assert_allclose(occ, ref, atol=1e-6)
    assert occ[10, 10, 10] == 1.0 and occ[10, 10 + 3, 10] == 0.0 and occ[10, 12, 10] == pytest.approx(0.5)


def test_rasterised_box_equals_region_of_larger_box():
    rng = synth.rng_for(9, 0)
    seg = synth.vessel_segments(rng, (40, 36, 32), 30, (0.5, 3.0))
    whole = synth.rasterize(seg, (0, 0, 0), (32, 36, 40))
    part = synth.rasterize(seg, (7, 5, 3), (20, 18, 16))  # origin (x, y, z), shape (z, y, x)
    np.testing.assert_array_equal(part, whole[3:23, 5:23, 7:23])


def test_milling_field_boxes_equal_regions_of_the_whole():
    f = synth.MillingField(extent_xyz=(48, 40, 36))
    whole = f.box((0, 0, 0), (36, 40, 48))
    part = f.box((9, 4, 6), (20, 24, 30))
    np.testing.assert_array_equal(part, whole[6:26, 4:28, 9:39])
    assert whole.dtype == np.uint8


def test_milling_stripes():
    # background 30 striped by 1 + 0.2 sin(2 pi z / 64): plane means 36 at z = 16, 24 at z = 48
    f = synth.MillingField(extent_xyz=(64, 64, 64), vessel_fraction=0.0)
    v = f.box((0, 0, 0), (64, 64, 64)).astype(np.float64)
    assert v[16].mean() - v[48].mean() == pytest.approx(12.0, abs=1.5)


def test_microct_bricks():
    specs = synth.brick_specs(n_bricks=16, extent_xyz=(512, 512, 512))
    for s in specs:
        assert all(64 <= c <= 192 for c in s.core_xyz)
        assert all(s.halo <= o and o + c + s.halo <= 512 for o, c in zip(s.origin_xyz, s.core_xyz))
    f = synth.MicroCTField(extent_xyz=(256, 256, 256))
    s = synth.BrickSpec((40, 50, 60), (30, 20, 25), 6)
    b1, b2 = f.brick(s, 2), f.brick(s, 2)
    assert b1.shape == (25 + 12, 20 + 12, 30 + 12) and b1.dtype == np.uint16
    np.testing.assert_array_equal(b1, b2)


def test_lightsheet_truth_is_half_occupancy_before_the_blur():
    vol, mask = synth.lightsheet_volume_u16((24, 28, 32), truth=True)
    rng = synth.rng_for(2, 0)
    n = max(8, int(round(2000 * (24 * 28 * 32) / 512 ** 3)))
    seg = synth.vessel_segments(rng, (32, 28, 24), n, (0.5, 3.0))
    occ = synth.rasterize(seg, (0, 0, 0), (24, 28, 32))
    np.testing.assert_array_equal(mask, occ >= 0.5)
    assert vol.dtype == np.uint16 and vol.shape == (24, 28, 32)


def test_mean_rule_phi0_slabs_equal_whole_volume_rule():
    vol = synth.tree_volume_u8((40, 24, 28), n_segments=10)
    m = ndi.uniform_filter(vol.astype(np.float64), size=3, mode="nearest")
    ref = np.where(m > vol.mean(dtype=np.float64), 2.0, -2.0).astype(np.float32)
    for slab in (7, 16, 64):
        np.testing.assert_array_equal(synth.mean_rule_phi0(vol, slab=slab), ref)


def test_serving_mix():
    specs = synth.serve_request_specs(200)
    for s in specs:
        assert s.sigma in (2.0, 3.0, 4.0, 6.0)
        assert s.halo == int(round(3 * s.sigma))
        assert all(32 <= c <= 256 for c in s.core_zyx)
        assert 50 <= s.iters <= 500
        assert s.padded_zyx == tuple(c + 2 * s.halo for c in s.core_zyx)
    assert {s.source for s in specs} == {"lightsheet", "microct", "milling"}
