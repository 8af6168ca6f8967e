"""Host buffers through the library's transfers.

Pinned host memory (page-locked by CUDA) is copied by the library's SM copy
kernels through its device mapping: 16-byte words when both addresses and the
size allow it, else 4-byte words, else bytes.  Pageable memory goes through
cudaMemcpyAsync.  Every form must give the device-buffer result bit for bit:
plain evolution, batch, serving, initialisation and isosurface extraction.
"""
import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = 4300.0
PARAMS = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pinned(a, offset=0):
    """A pinned host copy of `a` starting `offset` elements into its allocation."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    flat = torch.empty(t.numel() + offset, dtype=t.dtype).pin_memory()
    v = flat[offset:].view(t.shape)
    v.copy_(t)
    assert v.is_pinned()
    return v


# (24, 28, 36): sizes divisible by 16 bytes; (13, 17, 19): not (4- and 1-byte forms)
@pytest.mark.parametrize("shape", [(24, 28, 36), (13, 17, 19)])
@pytest.mark.parametrize("offset", [0, 1])
def test_evolve_with_pinned_buffers(ctx, shape, offset):
    vol = synth.lightsheet_volume_u16(shape)
    phi0 = synth.mean_rule_phi0(vol)
    ref = ctx.evolve(dev(vol), dev(phi0), PARAMS, 3).cpu().numpy()
    out = pinned(np.zeros_like(phi0), offset)
    got = ctx.evolve(pinned(vol, offset), pinned(phi0, offset), PARAMS, 3, out=out)
    np.testing.assert_array_equal(got.numpy(), ref)


def test_pageable_and_pinned_agree(ctx):
    vol = synth.lightsheet_volume_u16((20, 24, 28))
    phi0 = synth.mean_rule_phi0(vol)
    a = ctx.evolve(vol, phi0.copy(), PARAMS, 2)  # numpy: pageable
    b = ctx.evolve(pinned(vol), pinned(phi0), PARAMS, 2, out=pinned(np.zeros_like(phi0)))
    np.testing.assert_array_equal(a, b.numpy())


def test_batch_and_serve_with_pinned_buffers(ctx):
    specs = [(20, 24, 28), (13, 17, 19)]
    vols = [synth.lightsheet_volume_u16(s, brick=k) for k, s in enumerate(specs)]
    phis = [synth.mean_rule_phi0(v) for v in vols]
    ref = [ctx.evolve(dev(v), dev(p), PARAMS, 3).cpu().numpy() for v, p in zip(vols, phis)]
    items = [(pinned(v, k), pinned(p, k), PARAMS, 3, pinned(np.zeros_like(p), k))
             for k, (v, p) in enumerate(zip(vols, phis))]
    outs = ctx.evolve_batch(items)
    for o, r in zip(outs, ref):
        np.testing.assert_array_equal(o.numpy(), r)
    keep = [(pinned(v), pinned(p), pinned(np.zeros_like(p))) for v, p in zip(vols, phis)]
    tickets = [ctx.submit(hv, hp, PARAMS, 3, ho) for hv, hp, ho in keep]
    for t in tickets:
        ctx.wait(t, -1)
    for (_, _, ho), r in zip(keep, ref):
        np.testing.assert_array_equal(ho.numpy(), r)


def test_init_and_isosurface_from_pinned_buffers(ctx):
    vol = synth.lightsheet_volume_u16((24, 28, 36))
    phi_d, n_d = ctx.init_phi0(dev(vol), 1.5, 0.3, 2.0)
    phi_h, n_h = ctx.init_phi0(pinned(vol, 1), 1.5, 0.3, 2.0)
    assert n_d == n_h
    np.testing.assert_array_equal(phi_h.cpu().numpy(), phi_d.cpu().numpy())
    tri_d, key_d = ctx.isosurface(phi_d)
    tri_h, key_h = ctx.isosurface(pinned(phi_d.cpu().numpy(), 1))
    assert len(key_d) == len(key_h) > 0
    od, oh = np.argsort(key_d), np.argsort(key_h)
    np.testing.assert_array_equal(key_d[od], key_h[oh])
    np.testing.assert_array_equal(tri_d[od], tri_h[oh])
