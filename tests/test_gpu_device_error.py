"""The device-side failure path of the TMA copies, driven without a fault.

With RSF_OPT_FAULT_WAIT the z pass of group A arms its copy barriers for 16
bytes more than its TMA copies deliver, so that no barrier phase completes:
every bounded wait runs out (1 s, then 1 s more for the copies in flight), the
kernel records the expiry in the context's error word and returns.  The call
must fail with RSF_E_CUDA naming the expired wait, the context must stay in
error, and another context must be unaffected.
"""
import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(shape=(40, 36, 48)):
    vol = synth.tree_volume_u8(shape, brick=7, n_segments=6)
    phi0 = synth.box_phi0(shape, min(shape) // 2)
    p = dict(sigma=2.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)
    return vol, phi0, p


@pytest.mark.parametrize("form", ["li", "eq15"])
def test_expired_copy_wait_fails_the_call_and_spends_the_context(form):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol, phi0, p = _case()
    v = torch.from_numpy(vol).cuda()
    ph = torch.from_numpy(phi0).cuda()
    ctx = rsf.Context(0)
    try:
        ctx.set_force(form)
        ctx.set_option(rsf.OPT_FAULT_WAIT, 1)
        with pytest.raises(rsf.RSFError) as e:
            ctx.evolve(v, ph, p, 1)
        assert e.value.status == -3
        assert "bounded wait" in str(e.value)
        # the error word stays set: later calls on this context fail too
        ctx.set_option(rsf.OPT_FAULT_WAIT, 0)
        with pytest.raises(rsf.RSFError) as e2:
            ctx.evolve(v, ph, p, 1)
        assert e2.value.status == -3
    finally:
        ctx.close()
    # the GPU and other contexts are unaffected
    fresh = rsf.Context(0)
    try:
        fresh.set_force(form)
        out = fresh.evolve(v, ph, p, 2).cpu().numpy()
        assert np.isfinite(out).all()
    finally:
        fresh.close()
