"""No result depends on memory the iteration did not write.

With RSF_OPT_POISON every working field that an iteration must write before
it reads it (the intermediate fields, the second phi buffer, both buffers of
the Heaviside argument) starts as all-ones bytes -- a NaN in FP32, FP16 and
BF16.  Any read of an element no kernel wrote (a pitch column, a halo row, a
ragged tile edge, a stale slot) would carry NaN into phi or change it; the
poisoned runs must equal the clean ones bit for bit, on ragged shapes at
every instantiated radius, both force forms, FP32 and 16-bit storage, both
schedules, batches and served requests.  (The check stands in for a memory
sanitizer, which this pool does not run.)
"""
import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# ragged shapes: none a multiple of the 32-column pitch or of the tile heights
CASES = [((13, 17, 19), 3.0), ((21, 35, 33), 2.0), ((19, 26, 45), 4.0), ((23, 30, 37), 5.0), ((27, 29, 31), 6.0),
         ((9, 40, 70), 1.5), ((30, 12, 50), 2.5)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _inputs(k, shape):
    vol = synth.tree_volume_u8(shape, brick=300 + k, n_segments=8)
    return vol, synth.mean_rule_phi0(vol)


def _params(sigma):
    return dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    clean, poisoned = rsf.Context(0), rsf.Context(0)
    poisoned.set_option(rsf.OPT_POISON, 1)
    yield clean, poisoned
    clean.close()
    poisoned.close()


@pytest.mark.parametrize("path", ["auto", "passes"])
@pytest.mark.parametrize("form,storage", [("li", "f32"), ("li", "f16"), ("eq15", "f32"), ("eq15", "bf16")])
def test_plain_runs_read_only_written_memory(ctxs, path, form, storage):
    if path == "passes" and (form != "li" or storage != "f32"):
        pytest.skip("the six-pass schedule has FP32 storage and Li's form only")
    for c in ctxs:
        c.set_path(path)
        c.set_force(form)
        c.set_storage(storage)
    try:
        for k, (shape, sigma) in enumerate(CASES):
            vol, phi0 = _inputs(k, shape)
            p = _params(sigma)
            a = ctxs[0].evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
            b = ctxs[1].evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
            assert np.all(np.isfinite(b)), f"{shape} sigma {sigma}: NaN from unwritten memory"
            np.testing.assert_array_equal(b, a, err_msg=f"{shape} sigma {sigma}")
    finally:
        for c in ctxs:
            c.set_path("auto")
            c.set_force("li")
            c.set_storage("f32")


def test_batched_and_served_bricks_read_only_written_memory(ctxs):
    clean, poisoned = ctxs
    items_c, items_p, ref = [], [], []
    for k, (shape, sigma) in enumerate(CASES):
        vol, phi0 = _inputs(k, shape)
        p = _params(sigma)
        ref.append(clean.evolve(dev(vol), dev(phi0), p, 4).cpu().numpy())
        items_p.append((dev(vol), dev(phi0), p, 4))
    for o, r in zip(poisoned.evolve_batch(items_p), ref):
        assert np.all(np.isfinite(o.cpu().numpy()))
        np.testing.assert_array_equal(o.cpu().numpy(), r)
    served = rsf.Context(0)
    try:
        served.set_option(rsf.OPT_POISON, 1)
        outs, tickets = [], []
        for v, ph, p, it in items_p:
            o = torch.empty_like(ph)
            outs.append(o)
            tickets.append(served.submit(v, ph, p, it, o))
        for t in tickets:
            assert served.wait(t, 60000) == 0
        for o, r in zip(outs, ref):
            np.testing.assert_array_equal(o.cpu().numpy(), r)
    finally:
        served.close()
