"""Pins of the oracle's second data-term form: the paper's Eq. (15) with
sigma_2 = 0, its setting for the 3-D runs (Sec. 5.3).  With K(sigma_2) the
identity, F_+- = I^2 - 2 r_+- I + r_+-^2 = (I - r_+-)^2, r_+ = f_1, r_- = f_2.

* A brute-force numpy evaluation (explicit kernel offsets, explicit
  reflect-101 maps) agrees with the separable oracle step.
* The direct-sum voxel evaluation agrees with it, terms included.
* Constant phi: kappa = L = 0 and f_1 = f_2 = m = K*I / K*1, so the step is
  phi' = phi - dt delta(phi) (lambda1 - lambda2) (I - m)^2, with m from
  scipy's zero-padded correlation.
* The data terms are squares (>= 0) and vanish where the image is constant.
* The paper's 3-D parameter set segments a noisy ball (Dice >= 0.95).
"""
import json
import os

import numpy as np
import pytest

import oracle

ndi = pytest.importorskip("scipy.ndimage")

PARAMS_C1 = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def _brute_force_step_eq15(I, phi, p):
    g = oracle.taps(p["sigma"])
    R = (g.size - 1) // 2
    nz, ny, nx = I.shape

    def K(F):
        P = np.pad(F, R)
        out = np.zeros_like(F)
        for c in range(-R, R + 1):
            for b in range(-R, R + 1):
                for a in range(-R, R + 1):
                    out += g[a + R] * g[b + R] * g[c + R] * P[R + c:R + c + nz, R + b:R + b + ny, R + a:R + a + nx]
        return out

    eps = p["eps"]
    H = 0.5 * (1.0 + (2.0 / np.pi) * np.arctan(phi / eps))
    r_plus = K(H * I) / K(H)
    r_minus = K((1 - H) * I) / K(1 - H)
    F_plus = I * I - 2.0 * r_plus * I + r_plus * r_plus        # Eq. (15) with K(sigma_2) = identity
    F_minus = I * I - 2.0 * r_minus * I + r_minus * r_minus
    gg = p["lambda1"] * F_plus - p["lambda2"] * F_minus

    def m(i, n):
        return np.where(i < 0, -i, np.where(i >= n, 2 * (n - 1) - i, i))

    zi, yi, xi = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def at(F, dz, dy, dx):
        return F[m(zi + dz, nz), m(yi + dy, ny), m(xi + dx, nx)]

    gx = (at(phi, 0, 0, 1) - at(phi, 0, 0, -1)) / 2
    gy = (at(phi, 0, 1, 0) - at(phi, 0, -1, 0)) / 2
    gz = (at(phi, 1, 0, 0) - at(phi, -1, 0, 0)) / 2
    mag = np.sqrt(gx ** 2 + gy ** 2 + gz ** 2) + 1e-10
    nxf, nyf, nzf = gx / mag, gy / mag, gz / mag
    kap = ((at(nxf, 0, 0, 1) - at(nxf, 0, 0, -1)) + (at(nyf, 0, 1, 0) - at(nyf, 0, -1, 0))
           + (at(nzf, 1, 0, 0) - at(nzf, -1, 0, 0))) / 2
    lap = sum(at(phi, *o) for o in [(0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]) - 6 * phi
    delta = (eps / np.pi) / (eps * eps + phi * phi)
    return phi + p["dt"] * (p["mu"] * (lap - kap) + delta * (p["nu"] * kap - gg))


@pytest.mark.parametrize("shape,sigma,seed", [((6, 7, 8), 1.0, 31), ((7, 5, 9), 1.5, 32)])
def test_eq15_step_matches_brute_force(shape, sigma, seed):
    rng = np.random.default_rng(seed)
    I = rng.uniform(0, 255, size=shape)
    phi = rng.normal(0, 3, size=shape)
    p = dict(PARAMS_C1, sigma=sigma)
    ref = _brute_force_step_eq15(I, phi, p)
    out, dump = oracle.step(I, phi, p, dump=True, force="eq15")
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())
    for (z, y, x) in [(0, 0, 0), (shape[0] - 1, 2, shape[2] - 1), (3, 4, 5)]:
        v, t = oracle.point_next(I, phi, p, x, y, z, terms=True, force="eq15")
        assert abs(v - ref[z, y, x]) < 1e-9 * max(1.0, abs(ref[z, y, x]))
        for k in ("e1", "e2", "g", "kappa", "lap"):
            assert abs(t[k] - dump[k][z, y, x]) <= 1e-9 * max(1.0, abs(dump[k][z, y, x])), k
    # the two forms differ on such inputs
    assert np.abs(out - oracle.step(I, phi, p)).max() > 1e-3


def test_eq15_constant_phi_is_squared_deviation_from_local_mean():
    rng = np.random.default_rng(41)
    I = rng.uniform(0, 255, size=(8, 9, 10))
    phi = np.full(I.shape, -0.4)
    p = dict(PARAMS_C1, sigma=1.0)
    g = oracle.taps(1.0)
    K3 = g[:, None, None] * g[None, :, None] * g[None, None, :]
    KI = ndi.correlate(I, K3, mode="constant", cval=0.0)
    K1 = ndi.correlate(np.ones_like(I), K3, mode="constant", cval=0.0)
    mloc = KI / K1
    delta = (1.0 / np.pi) / (1.0 + 0.16)
    expect = -0.4 - p["dt"] * delta * (p["lambda1"] - p["lambda2"]) * (I - mloc) ** 2
    out = oracle.step(I, phi, p, force="eq15")
    np.testing.assert_allclose(out, expect, rtol=1e-11, atol=1e-9)


def test_eq15_terms_are_squares_and_vanish_on_constant_image():
    rng = np.random.default_rng(42)
    I = rng.uniform(0, 255, size=(9, 8, 7))
    phi = rng.normal(0, 2, size=I.shape)
    _, d = oracle.step(I, phi, PARAMS_C1, dump=True, force="eq15")
    assert d["e1"].min() >= 0.0 and d["e2"].min() >= 0.0
    _, d = oracle.step(np.full(I.shape, 77.0), phi, PARAMS_C1, dump=True, force="eq15")
    assert np.abs(d["g"]).max() < 1e-9


def test_eq15_noisy_ball_with_the_papers_3d_parameters():
    """Sec. 5.3: sigma_1 = 5, sigma_2 = 0, dt = 0.06, alpha = 255^2 * 0.0009, beta = 0.1."""
    p3 = json.load(open(GOLDEN))["params_3d"]
    assert float(p3["sigma2"]) == 0.0
    p = dict(sigma=float(p3["sigma1"]), eps=1.0, lambda1=float(p3["beta"]), lambda2=float(p3["beta"]),
             nu=float(p3["alpha"]), mu=1.0, dt=float(p3["dt"]))
    n, r = 40, 10.0
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    c = (n - 1) / 2.0
    rho = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    I = np.where(rho <= r, 200.0, 30.0) + np.random.default_rng(0).normal(0.0, 15.0, size=rho.shape)
    phi0 = np.full(I.shape, -2.0)
    lo, hi = int(c) - 5, int(c) + 7
    phi0[lo:hi, lo:hi, lo:hi] = 2.0
    phi = oracle.evolve(I, phi0, p, 60, omp=True, force="eq15")
    inside, ball = phi > 0, rho <= r
    dice = 2.0 * (inside & ball).sum() / (inside.sum() + ball.sum())
    assert dice >= 0.95, dice
