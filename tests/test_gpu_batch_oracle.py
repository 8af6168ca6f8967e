"""Batched and served bricks against the FP64 oracle.

Every brick of an rsf_evolve_batch call, and every request of a served mix,
is advanced k iterations; from the state reached, one more batched (or
served) iteration must match the oracle's step on that brick voxel by voxel
within the per-iteration bound of its storage: 1e-3 * c0 plus eight FP32
ulps of |phi| for FP32 storage; 2e-2 * c0, the ulps and four FP16 roundoffs
of the force magnitude (the stored fits enter the data terms relative to
their own size) for FP16.  Sign disagreement <= 1e-4 in both.  The bricks
mix shapes, radii (sigma 2-6), image types and both data-term forms, so each
batched launch covers bricks of several sizes at once.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import assert_phi_close, storage_force_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [  # (shape zyx, sigma, dtype, iterations before the checked step)
    ((37, 50, 29), 3.0, np.uint8, 6),
    ((48, 40, 64), 2.0, np.uint16, 9),
    ((20, 24, 28), 3.0, np.uint8, 3),
    ((45, 17, 33), 4.0, np.float32, 5),
    ((24, 40, 36), 2.0, np.uint16, 1),
    ((30, 34, 26), 6.0, np.uint8, 4),
]


def _brick(k, shape, sigma, dtype):
    rng = np.random.default_rng(300 + k)
    base = synth.tree_volume_u8(shape, brick=30 + k, n_segments=10).astype(np.float64)
    if dtype == np.uint16:
        vol, nu = (base * 16).astype(np.uint16), 0.004 * (255 * 16) ** 2
    elif dtype == np.float32:
        vol, nu = (base + rng.normal(0, 1, size=shape)).astype(np.float32), 0.004 * 255.0 ** 2
    else:
        vol, nu = base.astype(np.uint8), 0.004 * 255.0 ** 2
    phi0 = synth.box_phi0(shape, min(shape) // 2)
    return vol, phi0, dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=nu, mu=1.0, dt=0.1)


@pytest.fixture(scope="module")
def bricks():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return [_brick(k, *s[:3]) + (s[3],) for k, s in enumerate(SPECS)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(vol, phi_n, nxt, p, storage, form, what):
    ref, dump = oracle.step(vol.astype(np.float64), phi_n.astype(np.float64), p, dump=True, force=form)
    if storage == "f16" and form == "li":
        err = assert_phi_close(nxt, ref, phi_n, rel=2e-2, force=storage_force_tol(phi_n, dump, p, 2.0 ** -11),
                               what=what)
    else:
        err = assert_phi_close(nxt, ref, phi_n, rel=1e-3, what=what)
    print(f"{what}: max |dphi| {err:.3e}")


@pytest.mark.parametrize("form,storage", [("li", "f32"), ("li", "f16"), ("eq15", "f32")])
def test_batched_bricks_step_matches_oracle(bricks, form, storage):
    ctx = rsf.Context(0)
    try:
        ctx.set_force(form)
        ctx.set_storage(storage)
        ctx.set_option(rsf.OPT_AUTOTUNE, 1)
        vols = [dev(v) for v, _, _, _ in bricks]
        phis = ctx.evolve_batch([(v, dev(p0), p, k) for v, (_, p0, p, k) in zip(vols, bricks)])
        nxts = ctx.evolve_batch([(v, ph, p, 1) for v, ph, (_, _, p, _) in zip(vols, phis, bricks)])
        for i, ((vol, _, p, k), ph, nx) in enumerate(zip(bricks, phis, nxts)):
            _check(vol, ph.cpu().numpy(), nx.cpu().numpy(), p, storage, form,
                   f"batched brick {i} {vol.shape} sigma {p['sigma']} {form}/{storage}, step {k}")
    finally:
        ctx.close()


@pytest.mark.parametrize("form", ["li", "eq15"])
def test_served_mix_step_matches_oracle(bricks, form):
    """Requests submitted together (FP32 and FP16 storage in one mix): after k
    served iterations, one served iteration from each result against the oracle."""
    ctx = rsf.Context(0)
    try:
        ctx.set_force(form)
        storages = ["f32" if i % 2 == 0 or form == "eq15" else "f16" for i in range(len(bricks))]
        vols = [dev(v) for v, _, _, _ in bricks]
        mids = [torch.empty_like(dev(p0)) for _, p0, _, _ in bricks]
        t = [ctx.submit(v, dev(p0), p, k, m, storage=s)
             for v, (_, p0, p, k), m, s in zip(vols, bricks, mids, storages)]
        for tk in t:
            ctx.wait(tk, -1)
        nxts = [torch.empty_like(m) for m in mids]
        t = [ctx.submit(v, m, p, 1, o, storage=s) for v, m, (_, _, p, _), o, s in zip(vols, mids, bricks, nxts, storages)]
        for tk in t:
            ctx.wait(tk, -1)
        for i, ((vol, _, p, k), m, o, s) in enumerate(zip(bricks, mids, nxts, storages)):
            _check(vol, m.cpu().numpy(), o.cpu().numpy(), p, s, form,
                   f"served brick {i} {vol.shape} sigma {p['sigma']} {form}/{s}, step {k}")
    finally:
        ctx.close()
