"""rsf_evolve_curtain (the volume-level parallelism of Sec. 4.1) against the
oracle's curtain scheme and against the plain and batched GPU paths.

* GPU curtain vs oracle curtain, two iterations, within the FP32 bound.
* One sub-volume: the plain rsf_evolve result, bit for bit.
* Zero iterations: phi0 back (the normalised weights), to within an ulp.
* A voxel that only one sub-volume covers, away from its interior faces,
  carries that sub-volume's batched result bit for bit.
* Host pointers, aliasing and the argument checks.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import assert_phi_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    yield c
    c.close()


def _case(shape=(40, 44, 52), dtype=np.uint8):
    vol = synth.tree_volume_u8(shape, n_segments=16)
    phi0 = synth.mean_rule_phi0(vol)
    if dtype == np.uint16:
        vol = (vol.astype(np.uint16) * 16)
    return vol, phi0


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("edge,curtain,sigma", [(24, 4, 2.0), (20, 6, 1.5), (32, 8, 3.0)])
def test_curtain_matches_oracle(ctx, edge, curtain, sigma):
    vol, phi0 = _case()
    p = dict(synth.RSFParams().as_dict(), sigma=sigma)
    out = ctx.evolve_curtain(dev(vol), dev(phi0), p, 2, edge, curtain).cpu().numpy()
    ref = oracle.curtain_evolve(vol.astype(np.float64), phi0.astype(np.float64), p, 2, edge, curtain, omp=True)
    assert_phi_close(out, ref, phi0, what=f"curtain edge {edge} curtain {curtain}")


def test_single_subvolume_is_plain_evolve(ctx):
    vol, phi0 = _case()
    p = synth.RSFParams().as_dict()
    a = ctx.evolve_curtain(dev(vol), dev(phi0), p, 4, 64, 8).cpu().numpy()
    b = ctx.evolve(dev(vol), dev(phi0), p, 4).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_zero_iterations_give_phi0(ctx):
    vol, phi0 = _case()
    a = ctx.evolve_curtain(dev(vol), dev(phi0), synth.RSFParams().as_dict(), 0, 16, 4).cpu().numpy()
    np.testing.assert_allclose(a, phi0, rtol=2.0 ** -22, atol=0)


def test_interior_voxels_carry_the_subvolume_result(ctx):
    vol, phi0 = _case((36, 40, 60), np.uint16)
    p = dict(synth.RSFParams().as_dict(), nu=0.004 * (255 * 16) ** 2)
    edge, curtain, it = 32, 6, 3
    out = ctx.evolve_curtain(dev(vol), dev(phi0), p, it, edge, curtain).cpu().numpy()
    nz, ny, nx = vol.shape
    starts = [oracle.curtain_starts(n, edge, curtain) for n in (nz, ny, nx)]
    items, boxes = [], []
    for z0 in starts[0]:
        for y0 in starts[1]:
            for x0 in starts[2]:
                sl = np.s_[z0:z0 + edge, y0:y0 + edge, x0:x0 + edge]
                items.append((dev(vol[sl]), dev(phi0[sl]), p, it))
                boxes.append((z0, y0, x0))
    subs = [o.cpu().numpy() for o in ctx.evolve_batch(items)]
    count = np.zeros(vol.shape, dtype=int)
    for (z0, y0, x0) in boxes:
        count[z0:z0 + edge, y0:y0 + edge, x0:x0 + edge] += 1
    checked = 0
    for (z0, y0, x0), sub in zip(boxes, subs):
        sl = np.s_[z0:z0 + edge, y0:y0 + edge, x0:x0 + edge]
        one = count[sl] == 1
        # weight 1: at least `curtain` voxels from every interior face
        inner = np.ones(sub.shape, dtype=bool)
        for ax, (s, n) in enumerate(zip((z0, y0, x0), (nz, ny, nx))):
            idx = np.arange(min(edge, n))
            m = np.ones(idx.shape, dtype=bool)
            if s > 0:
                m &= idx >= curtain
            if s + edge < n:
                m &= idx < edge - curtain
            shape = [1, 1, 1]
            shape[ax] = idx.size
            inner &= m.reshape(shape)
        sel = one & inner
        np.testing.assert_array_equal(out[sl][sel], sub[sel])
        checked += int(sel.sum())
    assert checked > 1000


def test_host_pointers_and_alias(ctx):
    vol, phi0 = _case((30, 28, 36))
    p = synth.RSFParams().as_dict()
    ref = ctx.evolve_curtain(dev(vol), dev(phi0), p, 2, 16, 4).cpu().numpy()
    h = ctx.evolve_curtain(vol, phi0.copy(), p, 2, 16, 4)
    np.testing.assert_array_equal(h, ref)
    d = dev(phi0)
    ctx.evolve_curtain(dev(vol), d, p, 2, 16, 4, out=d)
    np.testing.assert_array_equal(d.cpu().numpy(), ref)


@pytest.mark.parametrize("edge,curtain", [(3, 1), (16, 0), (16, 9)])
def test_bad_arguments(ctx, edge, curtain):
    vol, phi0 = _case((20, 20, 20))
    with pytest.raises(rsf.RSFError) as e:
        ctx.evolve_curtain(dev(vol), dev(phi0), synth.RSFParams().as_dict(), 1, edge, curtain)
    assert e.value.status == -1


def test_curtain_eq15_f16_matches_oracle():
    """The context's force form applies inside the curtain scheme (16-bit storage
    leaves the Eq. (15) form's FP32 intermediates as they are)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol, phi0 = _case((36, 40, 44))
    p = dict(synth.RSFParams().as_dict(), sigma=2.0)
    c = rsf.Context(0)
    try:
        c.set_force("eq15")
        c.set_storage("f16")
        out = c.evolve_curtain(dev(vol), dev(phi0), p, 1, 24, 4).cpu().numpy()
    finally:
        c.close()
    ref = oracle.curtain_evolve(vol.astype(np.float64), phi0.astype(np.float64), p, 1, 24, 4, force="eq15")
    assert_phi_close(out, ref, phi0, rel=1e-3, sign_max=1e-4, what="curtain eq15")
