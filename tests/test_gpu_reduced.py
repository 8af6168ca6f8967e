"""16-bit storage of the intermediate fields (FP16, BF16) against the FP64 oracle.

(a, b) are stored in 16 bits with FP32 accumulation, the rounding residual of
each plane carried into the next plane of its column (noise shaping along z);
phi, the image, the x/y-convolved group-A pair, K*I and the x/y-convolved
(a, b) stay exact / FP32.  The gate, for both formats, is the per-iteration
bound for reduced storage: 2e-2 * c0, plus eight FP32 ulps of |phi|, plus four
unit roundoffs of the storage format (2^-11 for FP16, 2^-8 for BF16) times
the non-cancelled size of the force, dt * delta(phi_n) * (l1 |e1| + l2 |e2|):
the rounding of the stored fits enters the data terms relative to their own
size, and on 16-bit images those terms are ~(P/255)^2 larger than on 8-bit
ones.  Sign disagreement <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import assert_phi_close, paper_c1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _parity import storage_force_tol

REL = {"f16": 2e-2, "bf16": 2e-2}
UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
SIGN = {"f16": 1e-4, "bf16": 1e-4}


@pytest.fixture(scope="module", params=["f16", "bf16"])
def sctx(request):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    c.set_storage(request.param)
    c.storage = request.param
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [0, 5, 20])
def test_reduced_storage_per_iteration_c1(sctx, n):
    vol, phi0, p = paper_c1()
    v = dev(vol)
    phi_n = sctx.evolve(v, dev(phi0), p, n)
    nxt = sctx.evolve(v, phi_n, p, 1).cpu().numpy()
    phi_n = phi_n.cpu().numpy()
    ref, dump = oracle.step(vol.astype(np.float64), phi_n.astype(np.float64), p, dump=True)
    force = storage_force_tol(phi_n, dump, p, UNIT[sctx.storage])
    err = assert_phi_close(nxt, ref, phi_n, rel=REL[sctx.storage], force=force, sign_max=SIGN[sctx.storage],
                           what=f"{sctx.storage} step {n}->{n + 1}")
    print(f"{sctx.storage} step {n}: max |dphi| = {err:.3e}")


def test_reduced_storage_lightsheet_crop(sctx):
    vol = synth.lightsheet_volume_u16((48, 56, 64))
    phi0 = synth.mean_rule_phi0(vol)
    P = 4300.0
    p = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)
    v = dev(vol)
    for n in (0, 3):
        phi_n = sctx.evolve(v, dev(phi0), p, n)
        nxt = sctx.evolve(v, phi_n, p, 1).cpu().numpy()
        phi_n = phi_n.cpu().numpy()
        ref, dump = oracle.step(vol.astype(np.float64), phi_n.astype(np.float64), p, dump=True, omp=True)
        force = storage_force_tol(phi_n, dump, p, UNIT[sctx.storage])
        err = assert_phi_close(nxt, ref, phi_n, rel=REL[sctx.storage], force=force, sign_max=SIGN[sctx.storage],
                               what=f"{sctx.storage} light-sheet step {n}")
        print(f"{sctx.storage} light-sheet step {n}: max |dphi| = {err:.3e}")


def test_storage_needs_tiled_path():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    c.set_storage("f16")
    c.set_path("passes")
    vol, phi0, p = paper_c1()
    with pytest.raises(rsf.RSFError) as e:
        c.evolve(dev(vol), dev(phi0), p, 1)
    assert e.value.status == -1
    c.close()
