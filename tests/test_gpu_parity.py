"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

The gate is one iteration from a common state: the GPU's phi_{n+1} computed
from phi_n is compared voxel by voxel with the oracle's step from the same
phi_n, at several states along the GPU's own trajectory.  End to end, the
iteration map's own sensitivity (see test_oracle_dynamics) bounds what any
implementation that rounds differently can reach; the long-run check compares
against that envelope.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import C0, assert_phi_close, paper_c1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["auto", "passes"])
def ctx(request):
    """Every test runs on the default (tiled) schedule and on the six-pass one."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    c.set_path(request.param)
    c.path = request.param
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _f64(a):
    return np.asarray(a, dtype=np.float64)


# ----------------------------------------------------------- stage parity

def test_stages_one_iteration_c1(ctx):
    vol, phi0, p = paper_c1()
    nxt, st = ctx.step_stages(dev(vol), dev(phi0), p)
    ref, d = oracle.step(_f64(vol), _f64(phi0), p, dump=True)
    st = host(st)
    np.testing.assert_allclose(st[0], d["f1"], atol=2e-3, rtol=1e-5, err_msg="f1")
    np.testing.assert_allclose(st[1], d["f2"], atol=2e-3, rtol=1e-5, err_msg="f2")
    # g = l1 e1 - l2 e2: FP32 error bound of terms of size (l1 + l2) * (2 * 255)^2
    g_tol = 64 * 2.0 ** -24 * (p["lambda1"] + p["lambda2"]) * (2 * 255.0) ** 2
    np.testing.assert_allclose(st[2], d["g"], atol=g_tol, rtol=0, err_msg="g")
    np.testing.assert_allclose(st[3], d["kappa"], atol=1e-5, rtol=0, err_msg="kappa")
    np.testing.assert_allclose(st[4], d["lap"], atol=1e-5, rtol=0, err_msg="lap")
    assert_phi_close(host(nxt), ref, phi0, what="phi_1")


def test_stages_from_evolved_state_c1(ctx):
    vol, phi0, p = paper_c1()
    phi_n = host(ctx.evolve(dev(vol), dev(phi0), p, 10))
    nxt, st = ctx.step_stages(dev(vol), dev(phi_n), p)
    ref, d = oracle.step(_f64(vol), _f64(phi_n), p, dump=True)
    st = host(st)
    np.testing.assert_allclose(st[0], d["f1"], atol=2e-3, rtol=1e-5, err_msg="f1")
    np.testing.assert_allclose(st[1], d["f2"], atol=2e-3, rtol=1e-5, err_msg="f2")
    np.testing.assert_allclose(st[4], d["lap"], atol=1e-4, rtol=1e-6, err_msg="lap")
    assert_phi_close(host(nxt), ref, phi_n, what="phi_11")


# ------------------------------------------------ per-iteration parity gate

@pytest.mark.parametrize("n", [0, 1, 5, 20, 49])
def test_per_iteration_along_trajectory_c1(ctx, n):
    vol, phi0, p = paper_c1()
    v = dev(vol)
    phi_n = ctx.evolve(v, dev(phi0), p, n)
    nxt = ctx.evolve(v, phi_n, p, 1)
    phi_n = host(phi_n)
    ref = oracle.step(_f64(vol), _f64(phi_n), p)
    assert_phi_close(host(nxt), ref, phi_n, what=f"step {n}->{n + 1}")


def test_end_to_end_two_iterations_c1(ctx):
    vol, phi0, p = paper_c1()
    out = host(ctx.evolve(dev(vol), dev(phi0), p, 2))
    ref = oracle.evolve(_f64(vol), _f64(phi0), p, 2, omp=True)
    assert_phi_close(out, ref, phi0, what="2 iterations")


def test_end_to_end_50_within_oracle_sensitivity_envelope_c1(ctx):
    """After the workload's 50 iterations the GPU may differ from the oracle no more
    than the oracle differs from itself when its state is perturbed at FP32
    rounding level after the first iteration."""
    vol, phi0, p = paper_c1()
    out = host(ctx.evolve(dev(vol), dev(phi0), p, 50)).astype(np.float64)
    I = _f64(vol)
    ref = oracle.evolve(I, _f64(phi0), p, 50, omp=True)
    phi1 = oracle.evolve(I, _f64(phi0), p, 1, omp=True)
    rng = np.random.default_rng(0)
    pert = oracle.evolve(I, phi1 * (1.0 + 2.0 ** -24 * rng.standard_normal(phi1.shape)), p, 49, omp=True)
    d_gpu = np.mean(np.sign(out) != np.sign(ref))
    d_ref = np.mean(np.sign(pert) != np.sign(ref))
    assert d_gpu <= max(3.0 * d_ref, 1e-4), (d_gpu, d_ref)
    ins_g, ins_o = out > 0, ref > 0
    dice = 2.0 * (ins_g & ins_o).sum() / (ins_g.sum() + ins_o.sum())
    assert dice >= 0.98


# ------------------------------------------- shapes, dtypes, sigmas, edges

@pytest.mark.parametrize("shape,sigma,dtype", [
    ((29, 50, 37), 3.0, np.uint8),     # odd sizes, ragged tiles in every axis
    ((4, 4, 4), 1.0, np.uint8),        # the smallest volume
    ((5, 7, 130), 2.0, np.uint16),     # x beyond one 128-wide chunk with a 2-voxel tail
    ((12, 9, 11), 5.0, np.float32),    # kernel wider than the volume
    ((33, 20, 18), 6.0, np.uint8),     # sigma 6: 25 taps
    ((16, 17, 15), 1.5, np.uint16),
])
def test_one_iteration_shapes_dtypes_sigmas(ctx, shape, sigma, dtype):
    rng = np.random.default_rng(hash((shape, sigma)) % 2 ** 32)
    if dtype == np.float32:
        vol = rng.uniform(-50.0, 300.0, size=shape).astype(np.float32)
    else:
        hi = 255 if dtype == np.uint8 else 1000
        vol = rng.integers(0, hi + 1, size=shape).astype(dtype)
    phi = rng.normal(0.0, 2.0, size=shape).astype(np.float32)
    p = dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)
    vt = dev(vol)
    out = host(ctx.evolve(vt, dev(phi), p, 1))
    ref = oracle.step(_f64(vol), _f64(phi), p)
    assert_phi_close(out, ref, phi, what=f"{shape} sigma={sigma} {np.dtype(dtype).name}")


def test_host_and_device_pointers_agree_bitwise(ctx):
    vol, phi0, p = paper_c1()
    a = host(ctx.evolve(dev(vol), dev(phi0), p, 3))
    b = ctx.evolve(vol, phi0.copy(), p, 3)          # numpy host buffers
    np.testing.assert_array_equal(a, b)


def test_output_may_alias_input_and_zero_iterations_copy(ctx):
    vol, phi0, p = paper_c1()
    ref = host(ctx.evolve(dev(vol), dev(phi0), p, 2))
    ph = dev(phi0)
    out = ctx.evolve(dev(vol), ph, p, 2, out=ph)
    assert out.data_ptr() == ph.data_ptr()
    np.testing.assert_array_equal(host(ph), ref)
    z = host(ctx.evolve(dev(vol), dev(phi0), p, 0))
    np.testing.assert_array_equal(z, phi0)


def test_repeated_calls_are_deterministic(ctx):
    vol, phi0, p = paper_c1()
    a = host(ctx.evolve(dev(vol), dev(phi0), p, 5))
    b = host(ctx.evolve(dev(vol), dev(phi0), p, 5))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("bad", ["dims", "sigma_nan", "sigma_big", "iters", "eps", "dt"])
def test_invalid_arguments_are_rejected(ctx, bad):
    vol, phi0, p = paper_c1()
    p = dict(p)
    v, ph, iters = dev(vol), dev(phi0), 1
    if bad == "dims":
        v, ph = dev(vol[:3]), dev(phi0[:3])
    elif bad == "sigma_nan":
        p["sigma"] = float("nan")
    elif bad == "sigma_big":
        p["sigma"] = 9.0
    elif bad == "iters":
        iters = -1
    elif bad == "eps":
        p["eps"] = 0.0
    elif bad == "dt":
        p["dt"] = -0.1
    with pytest.raises(rsf.RSFError) as e:
        ctx.evolve(v, ph, p, iters)
    assert e.value.status == -1


# -------------------------------------------- 16-bit light-sheet workload

@pytest.mark.parametrize("sigma", [3.0, 5.0])
def test_lightsheet_crop_per_iteration(ctx, sigma):
    vol = synth.lightsheet_volume_u16((72, 80, 96))
    phi0 = synth.mean_rule_phi0(vol)
    P = 4300.0
    p = dict(sigma=sigma, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * P * P, mu=1.0, dt=0.1)
    v = dev(vol)
    for n in (0, 3):
        phi_n = ctx.evolve(v, dev(phi0), p, n)
        nxt = host(ctx.evolve(v, phi_n, p, 1))
        phi_n = host(phi_n)
        ref = oracle.step(_f64(vol), _f64(phi_n), p, omp=True)
        assert_phi_close(nxt, ref, phi_n, what=f"light-sheet sigma={sigma} step {n}")


# ------------------------------------------- far inside region 1 (huge phi)

@pytest.mark.parametrize("form", ["li", "eq15"])
def test_far_inside_region_one(ctx, form):
    """A 24^3 block at phi = 1e6 (1 - H ~ 3e-7, so K*(1-H) vanishes over whole
    windows): the step stays finite everywhere and within the per-iteration bound
    of the oracle (delta ~ 3e-13 there, so any fit of the empty complement region
    leaves phi unchanged to FP32 precision)."""
    if form == "eq15" and ctx.path == "passes":
        pytest.skip("the six-pass schedule has no Eq. (15) form")
    vol, _, p = paper_c1()
    vol = vol[:44, :48, :52]
    phi = synth.box_phi0(vol.shape, 20)
    phi[10:34, 12:36, 14:38] = 1e6
    ctx.set_force(form)
    try:
        nxt = host(ctx.evolve(dev(vol), dev(phi), p, 1))
    finally:
        ctx.set_force("li")
    assert np.all(np.isfinite(nxt))
    ref = oracle.step(_f64(vol), _f64(phi), p, force=form)
    assert_phi_close(nxt, ref, phi, what=f"phi = 1e6 block, {form}")
