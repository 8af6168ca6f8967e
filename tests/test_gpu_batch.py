"""Batched bricks: each brick evolved inside rsf_evolve_batch equals the same
brick evolved alone by rsf_evolve, bit for bit (the batched launches compute
every voxel with the same arithmetic in the same order), for uneven brick
sizes, mixed radii, image types and iteration counts."""
import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [  # (shape zyx, sigma, dtype, iters)
    ((37, 50, 29), 3.0, np.uint8, 7),
    ((48, 40, 64), 2.0, np.uint16, 10),
    ((20, 24, 28), 3.0, np.uint8, 3),
    ((45, 17, 33), 4.0, np.float32, 5),
    ((30, 30, 30), 3.0, np.uint8, 0),
    ((24, 40, 36), 2.0, np.uint16, 1),
    ((40, 33, 41), 3.0, np.uint8, 10),
]


def _brick(k, shape, sigma, dtype):
    rng = np.random.default_rng(100 + k)
    base = synth.tree_volume_u8(shape, brick=k, n_segments=10).astype(np.float64)
    if dtype == np.uint16:
        vol = (base * 16).astype(np.uint16)
        nu = 0.004 * (255 * 16) ** 2
    elif dtype == np.float32:
        vol = (base + rng.normal(0, 1, size=shape)).astype(np.float32)
        nu = 0.004 * 255.0 ** 2
    else:
        vol = base.astype(np.uint8)
        nu = 0.004 * 255.0 ** 2
    phi0 = synth.box_phi0(shape, min(shape) // 2)
    p = dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=nu, mu=1.0, dt=0.1)
    return vol, phi0, p


@pytest.fixture(scope="module")
def bricks():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return [_brick(k, *s[:3]) + (s[3],) for k, s in enumerate(SPECS)]


def _plain(ctx, bricks):
    return [ctx.evolve(torch.from_numpy(v).cuda(), torch.from_numpy(p0).cuda(), p, it).cpu().numpy()
            for v, p0, p, it in bricks]


@pytest.mark.parametrize("graph,autotune,storage", [(1, 0, "f32"), (0, 0, "f32"), (1, 1, "f32"), (1, 0, "f16")])
def test_batch_equals_plain_bitwise(bricks, graph, autotune, storage):
    ctx = rsf.Context(0)
    ctx.set_storage(storage)
    ref = _plain(ctx, bricks)
    ctx.set_option(rsf.OPT_GRAPH, graph)
    ctx.set_option(rsf.OPT_AUTOTUNE, autotune)
    items = [(torch.from_numpy(v).cuda(), torch.from_numpy(p0).cuda(), p, it) for v, p0, p, it in bricks]
    outs = ctx.evolve_batch(items)
    for k, (o, r) in enumerate(zip(outs, ref)):
        np.testing.assert_array_equal(o.cpu().numpy(), r, err_msg=f"brick {k}")
    ctx.close()


def test_batch_host_buffers_and_alias(bricks):
    ctx = rsf.Context(0)
    ref = _plain(ctx, bricks[:3])
    items = []
    for v, p0, p, it in bricks[:3]:
        ph = p0.copy()
        items.append((v, ph, p, it, ph))  # host buffers, output aliases phi0
    outs = ctx.evolve_batch(items)
    for k, (o, r) in enumerate(zip(outs, ref)):
        np.testing.assert_array_equal(o, r, err_msg=f"brick {k}")
    ctx.close()


def test_batch_rejects_bad_brick(bricks):
    ctx = rsf.Context(0)
    v, p0, p, it = bricks[0]
    bad = dict(p, sigma=9.0)
    with pytest.raises(rsf.RSFError) as e:
        ctx.evolve_batch([(torch.from_numpy(v).cuda(), torch.from_numpy(p0).cuda(), p, it),
                          (torch.from_numpy(v).cuda(), torch.from_numpy(p0).cuda(), bad, it)])
    assert e.value.status == -1 and "brick 1" in str(e.value)
    ctx.close()


def test_autotune_report_lists_each_group(bricks):
    """With RSF_OPT_AUTOTUNE the batch picks, per brick group, the x/y planes per CTA,
    the update kernel's z chunk and the brick order by timing; the report lists one
    entry per group with a choice from the candidate sets and a time no worse than the
    defaults' (the defaults are the first candidate).  The results stay bit-identical
    to rsf_evolve (test_batch_equals_plain_bitwise)."""
    ctx = rsf.Context(0)
    assert ctx.autotune_report() == []
    ctx.set_option(rsf.OPT_AUTOTUNE, 1)
    items = [(torch.from_numpy(v).cuda(), torch.from_numpy(p0).cuda(), p, it) for v, p0, p, it in bricks]
    ctx.evolve_batch(items)
    rep = ctx.autotune_report()
    groups = {(int(2 * p["sigma"] + 0.5), np.dtype(v.dtype).name) for v, _, p, it in bricks if it > 0}
    assert len(rep) == len(groups), rep
    for r in rep:
        assert r["xyp"] in (8, 16, 32) and r["zc"] >= 16 and r["order"] in ("largest", "smallest")
        assert 0 < r["ms"] <= r["default_ms"]
    ctx.close()
