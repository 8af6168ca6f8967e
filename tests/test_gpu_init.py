"""rsf_init_phi0 (the seed initialisation of Sec. 4.3) against the oracle.

* The blob response D matches the oracle's FP64 response (FP32 filters).
* The seed mask is the oracle's seed rule applied to the GPU's own FP32
  response, exactly (both sides take the integer decision on the same values),
  and agrees with the oracle's own seeds wherever the decision is not within
  the FP32 error of a tie.
* phi0 is r0 minus the exact distance to the GPU's seeds.
* A blob gives its centre; a volume without a bright blob is refused; the
  argument checks.
"""
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


def _run(ctx, vol, s, t, r0):
    v = torch.from_numpy(vol).cuda()
    seeds = torch.zeros(vol.shape, dtype=torch.uint8, device="cuda")
    resp = torch.empty(vol.shape, dtype=torch.float32, device="cuda")
    phi, n = ctx.init_phi0(v, s, t, r0, seeds=seeds, response=resp)
    return phi.cpu().numpy(), n, seeds.cpu().numpy().astype(bool), resp.cpu().numpy()


@pytest.mark.parametrize("shape,dtype,s,t", [((12, 40, 52), np.uint8, 1.5, 0.2), ((9, 37, 44), np.uint16, 2.0, 0.1),
                                             ((6, 33, 29), np.float32, 1.0, 0.3)])
def test_init_matches_oracle(ctx, shape, dtype, s, t):
    base = synth.tree_volume_u8(shape, n_segments=14)
    if dtype == np.uint16:
        vol = (base.astype(np.uint16) * 16 + 5).astype(np.uint16)
    elif dtype == np.float32:
        vol = base.astype(np.float32) + np.random.default_rng(1).normal(0, 1, size=shape).astype(np.float32)
    else:
        vol = base
    r0 = 2.0
    phi, n, seeds, resp = _run(ctx, vol, s, t, r0)
    ref = oracle.doh_response(vol.astype(np.float64), s)
    # response: same -inf pattern away from a vanishing Laplacian, values within FP32 filter error
    fin = np.isfinite(ref) & np.isfinite(resp)
    scale = np.abs(ref[fin]).max()
    np.testing.assert_allclose(resp[fin], ref[fin], rtol=0, atol=2e-5 * scale)
    mism = np.isfinite(ref) != np.isfinite(resp)
    assert mism.mean() < 1e-3
    if mism.any():  # only where the response itself is tiny (the Laplacian's sign is a near tie)
        assert np.nanmax(np.abs(np.where(np.isfinite(ref), ref, resp)[mism])) < 1e-3 * scale
    # seeds: the oracle's rule on the GPU's own response, exactly
    np.testing.assert_array_equal(seeds, oracle.seeds_from_response(resp.astype(np.float64), t))
    assert n == int(seeds.sum()) > 0
    # and the oracle's own seeds, except within FP32 error of a tie
    own = oracle.doh_seeds(vol.astype(np.float64), s, t)
    assert (own != seeds).mean() <= 2e-3
    # phi0 from the GPU's seeds
    want = oracle.seed_phi0(vol.shape, np.argwhere(seeds), r0)
    err = np.abs(phi.astype(np.float64) - want) / np.maximum(1.0, np.abs(want))
    assert err.max() <= 4e-7, f"phi0: worst relative error {err.max():.3e}"


def test_blob_centre(ctx):
    n = 40
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(n), indexing="ij")
    vol = (30 + 170 * np.exp(-((x - 21.0) ** 2 + (y - 17.0) ** 2) / (2 * 2.5 ** 2))).astype(np.float32)
    phi, cnt, seeds, _ = _run(ctx, vol, 2.0, 0.1, 3.0)
    assert cnt == 4 and np.argwhere(seeds).tolist() == [[k, 17, 21] for k in range(4)]
    assert abs(phi[0, 17, 21] - 3.0) < 1e-6 and abs(phi[3, 17, 25] - (3.0 - 4.0)) < 1e-6
    assert abs(phi[1, 20, 25] - (3.0 - 5.0)) < 1e-6


def test_no_blob_is_refused(ctx):
    vol = np.zeros((5, 16, 16), dtype=np.uint8)  # zero response everywhere: no slice has a positive maximum
    with pytest.raises(rsf.RSFError) as e:
        ctx.init_phi0(torch.from_numpy(vol).cuda(), 1.5, 0.1, 2.0)
    assert e.value.status == -1


@pytest.mark.parametrize("s,t,r0", [(0.0, 0.1, 2.0), (6.0, 0.1, 2.0), (1.5, 1.0, 2.0), (1.5, 0.1, 0.0)])
def test_bad_arguments(ctx, s, t, r0):
    vol = synth.tree_volume_u8((8, 16, 16), n_segments=4)
    with pytest.raises(rsf.RSFError) as e:
        ctx.init_phi0(torch.from_numpy(vol).cuda(), s, t, r0)
    assert e.value.status == -1


def test_host_arrays(ctx):
    vol = synth.tree_volume_u8((10, 36, 40), n_segments=10)
    phi_d, n_d, seeds_d, _ = _run(ctx, vol, 1.5, 0.2, 2.0)
    seeds = np.zeros(vol.shape, dtype=np.uint8)
    phi_h, n_h = ctx.init_phi0(vol, 1.5, 0.2, 2.0, seeds=seeds)
    assert n_h == n_d
    np.testing.assert_array_equal(seeds.astype(bool), seeds_d)
    np.testing.assert_array_equal(phi_h, phi_d)
