"""Checkpoint and resume: phi and the number of iterations done are the whole
state of the evolution (the image's statistics, K*1 and K*I are recomputed
from the volume), so splitting a run and resuming from its phi must give the
uninterrupted result bit for bit.

* rsf_evolve(n1) then rsf_evolve(n2) from its phi = rsf_evolve(n1 + n2), in
  both data-term forms and with FP32 and FP16 storage; the same for batches.
* rsf_suspend on a running served request: the ticket resolves SUSPENDED with
  phi after k iterations and k reported; resubmitting the remaining
  iterations gives the uninterrupted result.
* rsf_suspend on a request still in the queue: k = 0 and phi_out = phi0.
"""
import time

import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = 4300.0
PARAMS = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol = synth.lightsheet_volume_u16((36, 40, 44))
    return vol, synth.mean_rule_phi0(vol)


@pytest.mark.parametrize("form", ["li", "eq15"])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_split_evolution_equals_whole(case, form, storage):
    vol, phi0 = case
    ctx = rsf.Context(0)
    try:
        ctx.set_force(form)
        ctx.set_storage(storage)
        v = dev(vol)
        whole = ctx.evolve(v, dev(phi0), PARAMS, 12).cpu().numpy()
        part = ctx.evolve(v, dev(phi0), PARAMS, 5)
        np.testing.assert_array_equal(ctx.evolve(v, part, PARAMS, 7).cpu().numpy(), whole)
        a = ctx.evolve_batch([(v, dev(phi0), PARAMS, 4), (v, dev(phi0), PARAMS, 9)])
        b = ctx.evolve_batch([(v, a[0], PARAMS, 8), (v, a[1], PARAMS, 3)])
        for o in b:
            np.testing.assert_array_equal(o.cpu().numpy(), whole)
    finally:
        ctx.close()


def test_suspend_a_running_request_and_resume(case):
    vol, phi0 = case
    total = 20000  # four launches per iteration: far more than the 20 ms before the suspension
    whole = rsf.Context(0).evolve(dev(vol), dev(phi0), PARAMS, total).cpu().numpy()
    ctx = rsf.Context(0)
    try:
        v = dev(vol)
        out = torch.full_like(dev(phi0), float("nan"))
        t = ctx.submit(v, dev(phi0), PARAMS, total, out)
        time.sleep(0.05)
        done = ctx.suspend(t)
        assert ctx.wait(t, 60000) == rsf.RSF_SUSPENDED
        k = done.value  # iterations done (0 if the request was still queued on a slow start)
        assert 0 <= k < total
        assert np.all(np.isfinite(out.cpu().numpy()))
        out2 = torch.empty_like(out)
        t2 = ctx.submit(v, out, PARAMS, total - k, out2)
        assert ctx.wait(t2, 60000) == rsf.RSF_OK
        np.testing.assert_array_equal(out2.cpu().numpy(), whole)
        st = ctx.serve_stats()
        assert st["suspended"] == 1 and st["completed"] == 1
    finally:
        ctx.close()


def test_suspend_a_queued_request(case):
    vol, phi0 = case
    ctx = rsf.Context(0)
    try:
        ctx.set_option(rsf.OPT_SERVE_SLOTS, 1)  # one brick at a time: the second waits in the queue
        v = dev(vol)
        blocker_out = torch.empty_like(dev(phi0))
        t_block = ctx.submit(v, dev(phi0), PARAMS, 100000, blocker_out)
        ph = dev(phi0)
        out = torch.full_like(ph, float("nan"))
        t = ctx.submit(v, ph, PARAMS, 20, out)
        done = ctx.suspend(t)
        assert ctx.wait(t, 60000) == rsf.RSF_SUSPENDED
        assert done.value == 0
        np.testing.assert_array_equal(out.cpu().numpy(), phi0)
        ctx.cancel(t_block)
        with pytest.raises(rsf.RSFError) as e:
            ctx.wait(t_block, 60000)
        assert e.value.status == -7
    finally:
        ctx.close()


def test_suspend_unknown_ticket(case):
    ctx = rsf.Context(0)
    try:
        with pytest.raises(rsf.RSFError) as e:
            ctx.suspend(12345)
        assert e.value.status == -5
    finally:
        ctx.close()
