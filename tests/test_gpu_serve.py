"""The serving loop (rsf_submit / rsf_poll / rsf_wait / rsf_cancel).

Requests of different sizes, radii, storage and iteration counts are submitted
while others run; each result must equal rsf_evolve on the same brick with the
same storage, bit for bit (continuous batching changes when a brick's
iterations run, not how).  Failure handling is exercised on the host only:
cancellation, a request larger than the HBM budget, admission that waits for
memory, an injected set-up failure of one admission, and an injected failure
of one descriptor upload of the active set.
"""
import time

import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPECS = [  # (shape zyx, sigma, iters, storage)
    ((40, 36, 44), 3.0, 12, "f32"),
    ((24, 28, 20), 2.0, 30, "f32"),
    ((48, 40, 32), 4.0, 8, "f16"),
    ((30, 30, 30), 6.0, 5, "f32"),
    ((20, 20, 20), 3.0, 0, "f32"),
    ((36, 24, 52), 3.0, 20, "f16"),
    ((28, 44, 36), 2.0, 3, "f32"),
    ((32, 32, 32), 4.0, 16, "f32"),
]


def _case(k, shape, sigma):
    vol = synth.tree_volume_u8(shape, brick=200 + k, n_segments=10)
    phi0 = synth.box_phi0(shape, min(shape) // 2)
    p = dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)
    return vol, phi0, p


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def footprint(shape, storage_bytes=4):
    """Device bytes of one served brick: phi and q pairs, profiles, constants, and
    the intermediate fields at an x pitch rounded up to 32: the x/y-convolved
    group-A pair (8), (a, b) in the storage type, the x/y-convolved (a, b) (8)
    and K*I (4) per pitched voxel."""
    nz, ny, nx = shape
    n = nx * ny * nz
    np_ = ((nx + 31) // 32 * 32) * ny * nz
    return 16 * n + (8 + 2 * storage_bytes + 8 + 4) * np_ + 4 * 4096


@pytest.fixture(scope="module")
def cases():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return [_case(k, s[0], s[1]) + s[2:] for k, s in enumerate(SPECS)]


def _plain(cases):
    ctx = rsf.Context(0)
    out = []
    for vol, phi0, p, iters, storage in cases:
        ctx.set_storage(storage)
        out.append(ctx.evolve(dev(vol), dev(phi0), p, iters).cpu().numpy())
    ctx.close()
    return out


def test_served_results_equal_plain_in_the_mix(cases):
    ref = _plain(cases)
    ctx = rsf.Context(0)
    keep, tickets = [], []
    for k, (vol, phi0, p, iters, storage) in enumerate(cases):
        v, ph = dev(vol), dev(phi0)
        out = torch.full_like(ph, float("nan"))
        keep.append((v, ph, out))
        tickets.append(ctx.submit(v, ph, p, iters, out, storage=storage))
        time.sleep(0.002 * (k % 3))  # join while others are running
    for t in tickets:
        assert ctx.wait(t, 60000) == 0
    for k, ((v, ph, out), r) in enumerate(zip(keep, ref)):
        np.testing.assert_array_equal(out.cpu().numpy(), r, err_msg=f"request {k}")
    st = ctx.serve_stats()
    assert st["completed"] == len(cases) and st["failed"] == 0 and st["queued"] == 0
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"] <= st["latency_max_s"]
    with pytest.raises(rsf.RSFError) as e:  # a ticket is released by its final poll
        ctx.poll(tickets[0])
    assert e.value.status == -5
    ctx.close()


def test_cancel_and_host_buffers(cases):
    ctx = rsf.Context(0)
    vol, phi0, p, _, _ = cases[0]
    long_out = np.zeros_like(phi0)
    long_start = phi0.copy()
    t_long = ctx.submit(vol, long_start, p, 100000, long_out)  # host buffers
    time.sleep(0.05)
    ctx.cancel(t_long)
    with pytest.raises(rsf.RSFError) as e:
        ctx.wait(t_long, 60000)
    assert e.value.status == -7
    assert not long_out.any()  # a cancelled request does not write phi_out
    # the loop keeps serving after a cancellation
    out = np.zeros_like(phi0)
    start = phi0.copy()  # the caller keeps its buffers until the ticket resolves
    t = ctx.submit(vol, start, p, 4, out)
    assert ctx.wait(t, 60000) == 0
    ref = rsf.Context(0).evolve(vol, phi0.copy(), p, 4)
    np.testing.assert_array_equal(out, ref)
    ctx.close()


def test_over_budget_request_is_rejected(cases):
    vol, phi0, p, _, _ = cases[0]
    ctx = rsf.Context(0, hbm_budget_bytes=footprint(vol.shape) // 2)
    with pytest.raises(rsf.RSFError) as e:
        ctx.submit(dev(vol), dev(phi0), p, 3, dev(phi0))
    assert e.value.status == -2
    ctx.close()


def test_admission_waits_for_memory(cases):
    vol, phi0, p, _, _ = cases[1]  # 24 x 28 x 20
    budget = int(1.5 * footprint(vol.shape))  # room for one such brick at a time
    ctx = rsf.Context(0, hbm_budget_bytes=budget)
    ref = rsf.Context(0).evolve(dev(vol), dev(phi0), p, 6).cpu().numpy()
    outs, tickets = [], []
    v, ph = dev(vol), dev(phi0)
    for _ in range(4):
        o = torch.empty_like(ph)
        outs.append(o)
        tickets.append(ctx.submit(v, ph, p, 6, o))
    for t in tickets:
        assert ctx.wait(t, 60000) == 0
    for o in outs:
        np.testing.assert_array_equal(o.cpu().numpy(), ref)
    ctx.close()


def test_injected_admission_failure(cases):
    ctx = rsf.Context(0)
    ctx.set_option(rsf.OPT_FAULT_ADMISSION, 2)
    vol, phi0, p, _, _ = cases[6]
    ref = rsf.Context(0).evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
    v, ph = dev(vol), dev(phi0)
    outs = [torch.empty_like(ph) for _ in range(3)]
    tickets = [ctx.submit(v, ph, p, 3, o) for o in outs]
    statuses = []
    for t in tickets:
        try:
            statuses.append(ctx.wait(t, 60000))
        except rsf.RSFError as e:
            statuses.append(e.status)
    assert statuses == [0, -3, 0]
    np.testing.assert_array_equal(outs[0].cpu().numpy(), ref)
    np.testing.assert_array_equal(outs[2].cpu().numpy(), ref)
    st = ctx.serve_stats()
    assert st["failed"] == 1 and st["completed"] == 2
    ctx.close()


def test_injected_upload_failure(cases):
    """The first upload of the active set's launch descriptors fails on the host:
    the requests active at that tick resolve RSF_E_CUDA, with their phi_out left
    as it was; requests submitted afterwards are served normally."""
    ctx = rsf.Context(0)
    ctx.set_option(rsf.OPT_FAULT_UPLOAD, 1)
    vol, phi0, p, _, _ = cases[6]
    ref = rsf.Context(0).evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
    v, ph = dev(vol), dev(phi0)
    first = torch.full_like(ph, 7.0)
    t = ctx.submit(v, ph, p, 3, first)
    with pytest.raises(rsf.RSFError) as e:
        ctx.wait(t, 60000)
    assert e.value.status == -3
    assert bool((first == 7.0).all())
    later = torch.empty_like(ph)
    assert ctx.wait(ctx.submit(v, ph, p, 3, later), 60000) == 0
    np.testing.assert_array_equal(later.cpu().numpy(), ref)
    st = ctx.serve_stats()
    assert st["failed"] == 1 and st["completed"] == 1
    ctx.close()
