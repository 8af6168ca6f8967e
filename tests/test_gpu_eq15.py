"""GPU parity of the paper's own data-term form, Eq. (15) with sigma_2 = 0
(e_i = (I - f_i)^2; the group-B convolutions drop out), against the oracle's
same form: stages after one iteration, one iteration from common states along
the GPU's trajectory, the paper's 3-D parameter set (Sec. 5.3), batched and
served bricks equal to plain ones bit for bit, and the six-pass schedule
refusing the form.

Every check uses the base FP32 gate (1e-3 * c0 plus eight FP32 ulps of |phi|,
sign disagreement <= 1e-4): the form convolves both sides of Eq. (10)
directly, so each fit is a ratio of sums of non-negative weights.  Its
intermediates are FP32 whatever the storage option, so the FP16 and BF16
contexts must give the FP32 result bit for bit.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import assert_phi_close, paper_c1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _paper_3d_params():
    p = json.load(open(GOLDEN))["params_3d"]
    return dict(sigma=float(p["sigma1"]), eps=1.0, lambda1=float(p["beta"]), lambda2=float(p["beta"]),
                nu=float(p["alpha"]), mu=1.0, dt=float(p["dt"]))


@pytest.fixture(scope="module")
def ectx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    c.set_force("eq15")
    c.storage = "f32"
    yield c
    c.close()


def _check(ctx, vol, phi_n, nxt, p, what):
    ref = oracle.step(_f64(vol), _f64(phi_n), p, omp=True, force="eq15")
    err = assert_phi_close(nxt, ref, phi_n, rel=1e-3, sign_max=1e-4, what=f"eq15 {what}")
    print(f"eq15 {what}: max |dphi| {err:.3e}, sign disagreement {np.mean(np.sign(nxt) != np.sign(ref)):.2e}")
    return err


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_eq15_storage_option_changes_nothing(ectx, storage):
    vol = synth.lightsheet_volume_u16((40, 48, 72))
    phi0 = synth.mean_rule_phi0(vol)
    P = 4300.0
    p = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)
    ref = ectx.evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
    c = rsf.Context(0)
    try:
        c.set_force("eq15")
        c.set_storage(storage)
        out = c.evolve(dev(vol), dev(phi0), p, 3).cpu().numpy()
    finally:
        c.close()
    np.testing.assert_array_equal(out, ref)


def test_eq15_stages_one_iteration_c1(ectx):
    vol, phi0, p = paper_c1()
    nxt, st = ectx.step_stages(dev(vol), dev(phi0), p)
    ref, d = oracle.step(_f64(vol), _f64(phi0), p, dump=True, force="eq15")
    st = st.cpu().numpy()
    np.testing.assert_allclose(st[0], d["f1"], atol=2e-3, rtol=1e-5, err_msg="f1")
    np.testing.assert_allclose(st[1], d["f2"], atol=2e-3, rtol=1e-5, err_msg="f2")
    g_tol = 64 * 2.0 ** -24 * (p["lambda1"] + p["lambda2"]) * (2 * 255.0) ** 2
    np.testing.assert_allclose(st[2], d["g"], atol=g_tol, rtol=0, err_msg="g")
    np.testing.assert_allclose(st[3], d["kappa"], atol=1e-5, rtol=0, err_msg="kappa")
    np.testing.assert_allclose(st[4], d["lap"], atol=1e-5, rtol=0, err_msg="lap")
    assert_phi_close(nxt.cpu().numpy(), ref, phi0, what="eq15 phi_1")


@pytest.mark.parametrize("n", [0, 5, 20])
def test_eq15_per_iteration_c1(ectx, n):
    vol, phi0, p = paper_c1()
    v = dev(vol)
    phi_n = ectx.evolve(v, dev(phi0), p, n)
    nxt = ectx.evolve(v, phi_n, p, 1).cpu().numpy()
    _check(ectx, vol, phi_n.cpu().numpy(), nxt, p, f"step {n}")


def test_eq15_papers_3d_parameters(ectx):
    """sigma_1 = 5, sigma_2 = 0, dt = 0.06, alpha = 255^2 * 0.0009, beta = 0.1 (Sec. 5.3)."""
    vol = synth.tree_volume_u8((48, 56, 40))
    phi0 = synth.mean_rule_phi0(vol)
    p = _paper_3d_params()
    v = dev(vol)
    for n in (0, 10):
        phi_n = ectx.evolve(v, dev(phi0), p, n)
        nxt = ectx.evolve(v, phi_n, p, 1).cpu().numpy()
        _check(ectx, vol, phi_n.cpu().numpy(), nxt, p, f"paper 3-D parameters step {n}")


def test_eq15_lightsheet_crop(ectx):
    vol = synth.lightsheet_volume_u16((40, 48, 72))
    phi0 = synth.mean_rule_phi0(vol)
    P = 4300.0
    p = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)
    v = dev(vol)
    for n in (0, 3):
        phi_n = ectx.evolve(v, dev(phi0), p, n)
        nxt = ectx.evolve(v, phi_n, p, 1).cpu().numpy()
        _check(ectx, vol, phi_n.cpu().numpy(), nxt, p, f"light-sheet step {n}")


def test_eq15_batch_and_serve_equal_plain(ectx):
    specs = [((37, 50, 29), 3.0, 6), ((48, 40, 64), 2.0, 9), ((20, 24, 28), 5.0, 3)]
    items, ref = [], []
    for k, (shape, sigma, iters) in enumerate(specs):
        vol = synth.tree_volume_u8(shape, brick=k, n_segments=10)
        phi0 = synth.box_phi0(shape, min(shape) // 2)
        p = dict(synth.RSFParams().as_dict(), sigma=sigma)
        ref.append(ectx.evolve(dev(vol), dev(phi0), p, iters).cpu().numpy())
        items.append((dev(vol), dev(phi0), p, iters))
    outs = ectx.evolve_batch(items)
    for k, (o, r) in enumerate(zip(outs, ref)):
        np.testing.assert_array_equal(o.cpu().numpy(), r, err_msg=f"batched brick {k}")
    tickets, outs = [], []
    for v, p0, p, it in items:
        o = torch.empty_like(p0)
        outs.append(o)
        tickets.append(ectx.submit(v, p0, p, it, o, storage="f32"))
    for t in tickets:
        ectx.wait(t, -1)
    for k, (o, r) in enumerate(zip(outs, ref)):
        np.testing.assert_array_equal(o.cpu().numpy(), r, err_msg=f"served brick {k}")


def test_eq15_needs_the_tiled_path():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol, phi0, p = paper_c1()
    c = rsf.Context(0)
    try:
        c.set_force("eq15")
        c.set_path("passes")
        with pytest.raises(rsf.RSFError) as e:
            c.evolve(dev(vol), dev(phi0), p, 1)
        assert e.value.status == -1
    finally:
        c.close()
