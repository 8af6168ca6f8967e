"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one oracle function to a closed form, a library routine
(scipy.ndimage, numpy.gradient), a brute-force evaluation on a tiny volume,
or an exact invariance of the method, so that a dropped term, a wrong sign,
a wrong index or stride, or a transposed axis fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle

scipy_ndimage = pytest.importorskip("scipy.ndimage")

PARAMS_C1 = dict(sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1)
# The 3D parameter set of the paper's Monte-Carlo validation (Sec. 5.3):
# sigma_1 = 5, dt = 0.06, alpha = 255^2 * 0.0009 (-> nu), beta = 0.1 (-> lambda1 = lambda2).
PARAMS_PAPER3D = dict(sigma=5.0, eps=1.0, lambda1=0.1, lambda2=0.1, nu=255.0 ** 2 * 0.0009, mu=1.0, dt=0.06)


def _rand(shape, seed, lo=0.0, hi=255.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


# ------------------------------------------------------------------ taps (Eq. 7)

@pytest.mark.parametrize("sigma,R", [(1.0, 2), (2.0, 4), (3.0, 6), (4.0, 8), (5.0, 10), (6.0, 12),
                                     (2.25, 5), (0.75, 2), (1.2, 2)])
def test_radius_is_round_two_sigma(sigma, R):
    # R = round(2 sigma), halves away from zero: sigma=3 gives the 13-tap kernel.
    assert oracle.radius(sigma) == R
    assert oracle.taps(sigma).shape == (2 * R + 1,)


@pytest.mark.parametrize("sigma", [1.0, 3.0, 5.0, 6.0])
def test_taps_normalised_symmetric_gaussian(sigma):
    g = oracle.taps(sigma)
    R = (g.size - 1) // 2
    assert abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(g, g[::-1])
    k = np.arange(-R, R + 1)
    ratio = g / g[R]
    np.testing.assert_allclose(ratio, np.exp(-k * k / (2.0 * sigma * sigma)), rtol=1e-14)


# ---------------------------------------------------------------- conv (Eq. 6)

def _kernel3(g):
    return g[:, None, None] * g[None, :, None] * g[None, None, :]


@pytest.mark.parametrize("shape,sigma,seed", [((5, 6, 7), 1.0, 1), ((9, 7, 12), 1.5, 2), ((12, 11, 10), 2.0, 3),
                                              ((6, 13, 5), 3.0, 4)])
def test_conv_matches_library_direct_3d(shape, sigma, seed):
    """Separable x->y->z passes == scipy's direct 3-D correlation with zero padding."""
    F = _rand(shape, seed, -3.0, 5.0)
    g = oracle.taps(sigma)
    ref = scipy_ndimage.correlate(F, _kernel3(g), mode="constant", cval=0.0)
    np.testing.assert_allclose(oracle.conv3(F, sigma), ref, rtol=1e-12, atol=1e-12)


def test_conv_brute_force_offsets_non_cubic():
    """Explicit triple sum over kernel offsets, zero outside, on a non-cubic volume."""
    F = _rand((6, 8, 11), 7, -1.0, 1.0)
    sigma = 1.0
    g = oracle.taps(sigma)
    R = (g.size - 1) // 2
    nz, ny, nx = F.shape
    P = np.pad(F, R)
    ref = np.zeros_like(F)
    for c in range(-R, R + 1):
        for b in range(-R, R + 1):
            for a in range(-R, R + 1):
                w = g[a + R] * g[b + R] * g[c + R]
                ref += w * P[R + c:R + c + nz, R + b:R + b + ny, R + a:R + a + nx]
    np.testing.assert_allclose(oracle.conv3(F, sigma), ref, rtol=1e-12, atol=1e-14)


def test_conv_linear_and_impulse_response():
    sigma = 2.0
    g = oracle.taps(sigma)
    R = (g.size - 1) // 2
    A = _rand((11, 12, 13), 11, -1, 1)
    B = _rand((11, 12, 13), 12, -1, 1)
    np.testing.assert_allclose(oracle.conv3(2.0 * A - 3.0 * B, sigma),
                               2.0 * oracle.conv3(A, sigma) - 3.0 * oracle.conv3(B, sigma), atol=1e-13)
    # a delta away from the faces returns the 3-D kernel itself (a correlation of a symmetric kernel)
    D = np.zeros((2 * R + 3, 2 * R + 5, 2 * R + 7))
    cz, cy, cx = R + 1, R + 2, R + 3
    D[cz, cy, cx] = 1.0
    out = oracle.conv3(D, sigma)
    np.testing.assert_allclose(out[cz - R:cz + R + 1, cy - R:cy + R + 1, cx - R:cx + R + 1], _kernel3(g), atol=1e-17)
    assert abs(out.sum() - 1.0) < 1e-14


def test_k1_edge_profile():
    """K*1 is 1 at >= R from every face and (sum_{k>=0} g_k)^3 at a corner (zero padding)."""
    sigma = 3.0
    g = oracle.taps(sigma)
    R = (g.size - 1) // 2
    K1 = oracle.conv3(np.ones((2 * R + 4, 2 * R + 5, 2 * R + 6)), sigma)
    inner = K1[R:-R, R:-R, R:-R]
    np.testing.assert_allclose(inner, 1.0, atol=1e-14)
    half = g[R:].sum()
    assert abs(K1[0, 0, 0] - half ** 3) < 1e-14
    assert abs(K1[0, R + 1, R + 1] - half) < 1e-14  # one face only
    # separable profile: K1(x, y, z) = p(x) p(y) p(z)
    n = K1.shape
    p = [np.array([g[max(0, R - i):R + (m - i)].sum() for i in range(m)]) for m in n]
    np.testing.assert_allclose(K1, p[0][:, None, None] * p[1][None, :, None] * p[2][None, None, :], atol=1e-14)


# ------------------------------------------------------- H and delta (Eqs. 10, 14)

def test_heaviside_closed_forms():
    for eps in (1.0, 0.5, 2.0):
        assert oracle.heaviside(0.0, eps) == 0.5
        assert abs(oracle.heaviside(eps, eps) - 0.75) < 1e-15      # atan(1) = pi/4
        assert abs(oracle.heaviside(-eps, eps) - 0.25) < 1e-15
        assert abs(oracle.heaviside(math.sqrt(3) * eps, eps) - (0.5 + 1.0 / 3.0)) < 1e-15  # atan(sqrt 3) = pi/3
        assert oracle.heaviside(1e12, eps) > 1 - 1e-12
        assert oracle.heaviside(-1e12, eps) < 1e-12
        u = np.linspace(-5, 5, 41)
        np.testing.assert_allclose(oracle.heaviside(u, eps) + oracle.heaviside(-u, eps), 1.0, atol=1e-15)


def test_dirac_is_derivative_of_heaviside():
    for eps in (1.0, 0.3):
        assert abs(oracle.dirac(0.0, eps) - 1.0 / (math.pi * eps)) < 1e-15
        u = np.linspace(-6, 6, 25)
        h = 1e-5
        fd = (oracle.heaviside(u + h, eps) - oracle.heaviside(u - h, eps)) / (2 * h)
        np.testing.assert_allclose(oracle.dirac(u, eps), fd, rtol=1e-8, atol=1e-12)


# ----------------------------------------------------------- stencils (Eqs. 3-4)

def test_curvature_of_sphere_sdf_is_two_over_rho():
    n = 64
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    c = (n - 1) / 2.0
    rho = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi = rho - 16.0
    kap, lap = oracle.stencils(phi)
    sel = (rho >= 8) & (rho <= 24)
    rel = np.abs(kap[sel] - 2.0 / rho[sel]) * rho[sel] / 2.0
    assert rel.max() < 0.02
    # |grad phi| = 1 for an exact SDF, so the Laplacian equals the curvature there
    # and R(phi) = L phi - kappa vanishes up to discretisation error
    assert np.abs(lap[sel] - kap[sel]).max() < 0.02 * (2.0 / 8.0)


def test_curvature_and_laplacian_vs_numpy_gradient_interior():
    phi = np.random.default_rng(5).normal(size=(10, 12, 14))
    gz, gy, gx = np.gradient(phi)
    m = np.sqrt(gx * gx + gy * gy + gz * gz) + 1e-10
    k_ref = (np.gradient(gx / m, axis=2) + np.gradient(gy / m, axis=1) + np.gradient(gz / m, axis=0))
    l_ref = sum(np.roll(phi, s, axis=a) for a in range(3) for s in (1, -1)) - 6 * phi
    kap, lap = oracle.stencils(phi)
    I = (slice(2, -2),) * 3
    np.testing.assert_allclose(kap[I], k_ref[I], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(lap[I], l_ref[I], rtol=1e-12, atol=1e-12)


def test_laplacian_exact_on_quadratic_and_zero_on_linear():
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(10.0), np.arange(11.0), indexing="ij")
    _, lap = oracle.stencils(x * x + 2 * y * y - z * z + 3 * x * y)
    np.testing.assert_allclose(lap[1:-1, 1:-1, 1:-1], 2.0 + 4.0 - 2.0, atol=1e-11)
    kap, lap = oracle.stencils(0.3 * x - 0.2 * y + 0.5 * z)
    np.testing.assert_allclose(lap[1:-1, 1:-1, 1:-1], 0.0, atol=1e-12)
    np.testing.assert_allclose(kap[2:-2, 2:-2, 2:-2], 0.0, atol=1e-12)


def test_stencil_boundary_is_reflect101():
    """At the faces the stencils read through numpy's 'reflect' padding (reflect-101:
    the edge voxel is not repeated), applied to phi and, for the divergence, to the
    unit normal itself."""
    phi = np.random.default_rng(9).normal(size=(5, 6, 7))
    kap, lap = oracle.stencils(phi)
    P = np.pad(phi, 1, mode="reflect")
    c = (slice(1, -1),) * 3

    def sh(F, a, s):
        sl = list(c)
        sl[a] = slice(1 + s, F.shape[a] - 1 + s)
        return F[tuple(sl)]

    lap_ref = sum(sh(P, a, 1) + sh(P, a, -1) for a in range(3)) - 6 * phi
    np.testing.assert_allclose(lap, lap_ref, atol=1e-12)
    grad = [(sh(P, a, 1) - sh(P, a, -1)) / 2 for a in range(3)]  # axis order z, y, x
    mag = np.sqrt(sum(q * q for q in grad)) + 1e-10
    kap_ref = 0.0
    for a in range(3):
        Np = np.pad(grad[a] / mag, 1, mode="reflect")
        kap_ref = kap_ref + (sh(Np, a, 1) - sh(Np, a, -1)) / 2
    np.testing.assert_allclose(kap, kap_ref, atol=1e-12)
    # consequence of the index map: the normal's own-axis difference vanishes on that face
    assert np.all(np.isfinite(kap))


# ---------------------------------------------------------- local fits (Eq. 6)

def test_two_phase_fits_are_phase_values():
    """Piecewise-constant two-phase I with |phi| >> eps: f1 = a wherever the kernel
    meets the phi>0 phase, f2 = b wherever it meets the other phase."""
    rng = np.random.default_rng(3)
    shape = (14, 15, 16)
    mask = rng.random(shape) < 0.4
    a, b = 200.0, 30.0
    I = np.where(mask, a, b)
    phi = np.where(mask, 1e12, -1e12)
    _, d = oracle.step(I, phi, dict(PARAMS_C1, sigma=1.0), dump=True)
    np.testing.assert_allclose(d["f1"], a, rtol=1e-9)
    np.testing.assert_allclose(d["f2"], b, rtol=1e-9)


def test_constant_image_gives_zero_force():
    I = np.full((8, 9, 10), 77.0)
    phi = np.random.default_rng(4).normal(0, 2, size=I.shape)
    _, d = oracle.step(I, phi, PARAMS_C1, dump=True)
    np.testing.assert_allclose(d["f1"], 77.0, rtol=1e-13)
    np.testing.assert_allclose(d["f2"], 77.0, rtol=1e-13)
    for k in ("e1", "e2", "g"):
        assert np.abs(d[k]).max() < 1e-7


# -------------------------------------------------------- whole step (Eqs. 1, 13)

def _brute_force_step(I, phi, p):
    """Direct evaluation from the definitions with explicit loops over kernel offsets
    and explicit reflect-101 index maps (numpy only)."""
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
    f1 = K(H * I) / K(H)
    f2 = K((1 - H) * I) / K(1 - H)
    K1 = K(np.ones_like(I))
    e1 = K1 * I * I - 2 * I * K(f1) + K(f1 * f1)
    e2 = K1 * I * I - 2 * I * K(f2) + K(f2 * f2)
    gg = p["lambda1"] * e1 - p["lambda2"] * e2

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


@pytest.mark.parametrize("shape,sigma,seed", [((6, 7, 8), 1.0, 21), ((7, 5, 9), 1.5, 22)])
def test_step_matches_brute_force(shape, sigma, seed):
    rng = np.random.default_rng(seed)
    I = rng.uniform(0, 255, size=shape)
    phi = rng.normal(0, 3, size=shape)
    p = dict(PARAMS_C1, sigma=sigma)
    ref = _brute_force_step(I, phi, p)
    out = oracle.step(I, phi, p)
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())
    # the voxel-at-a-time evaluation with direct sums agrees as well
    for (z, y, x) in [(0, 0, 0), (shape[0] - 1, 2, shape[2] - 1), (3, 4, 5)]:
        assert abs(oracle.point_next(I, phi, p, x, y, z) - ref[z, y, x]) < 1e-9 * max(1.0, abs(ref[z, y, x]))
    # and its intermediate terms equal the separable step's stage fields
    _, dump = oracle.step(I, phi, p, dump=True)
    for (z, y, x) in [(0, 0, 0), (3, 4, 5)]:
        _, t = oracle.point_next(I, phi, p, x, y, z, terms=True)
        for k in ("e1", "e2", "g", "kappa", "lap"):
            assert abs(t[k] - dump[k][z, y, x]) <= 1e-9 * max(1.0, abs(dump[k][z, y, x])), k


def test_step_constant_phi_reduces_to_force_only():
    """phi constant: kappa = 0, L = 0, H cancels so f1 = f2 = K*I / K*1 and
    phi' = phi - dt delta(phi) (lambda1 - lambda2) e with e evaluated per voxel."""
    rng = np.random.default_rng(8)
    I = rng.uniform(0, 255, size=(7, 8, 9))
    phi = np.full(I.shape, 0.7)
    p = dict(PARAMS_C1, sigma=1.0)
    g = oracle.taps(1.0)
    K3 = _kernel3(g)
    nz, ny, nx = I.shape
    out = oracle.step(I, phi, p)

    def conv_at(F, z, y, x):
        s = 0.0
        for c in range(-2, 3):
            for b in range(-2, 3):
                for a in range(-2, 3):
                    if 0 <= z + c < nz and 0 <= y + b < ny and 0 <= x + a < nx:
                        s += K3[c + 2, b + 2, a + 2] * F(z + c, y + b, x + a)
        return s

    delta = (1.0 / np.pi) / (1.0 + 0.49)
    for (z, y, x) in [(0, 0, 0), (3, 4, 4), (6, 7, 8), (2, 0, 5)]:
        def f(zz, yy, xx):
            return conv_at(lambda a, b, c: I[a, b, c], zz, yy, xx) / conv_at(lambda a, b, c: 1.0, zz, yy, xx)
        K1 = conv_at(lambda a, b, c: 1.0, z, y, x)
        Kf = conv_at(f, z, y, x)
        Kf2 = conv_at(lambda a, b, c: f(a, b, c) ** 2, z, y, x)
        e = K1 * I[z, y, x] ** 2 - 2 * I[z, y, x] * Kf + Kf2
        expect = 0.7 - p["dt"] * delta * (p["lambda1"] - p["lambda2"]) * e
        assert abs(out[z, y, x] - expect) < 1e-9 * max(1.0, abs(expect))


def test_step_axis_permutation_and_mirror_equivariance():
    rng = np.random.default_rng(10)
    shape = (9, 10, 11)
    I = rng.uniform(0, 255, size=shape)
    phi = rng.normal(0, 2, size=shape)
    p = dict(PARAMS_C1, sigma=1.5)
    base = oracle.step(I, phi, p)
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        out = oracle.step(np.transpose(I, perm), np.transpose(phi, perm), p)
        np.testing.assert_allclose(out, np.transpose(base, perm), rtol=1e-11, atol=1e-10)
    for ax in range(3):
        out = oracle.step(np.flip(I, ax), np.flip(phi, ax), p)
        np.testing.assert_allclose(out, np.flip(base, ax), rtol=1e-11, atol=1e-10)


def test_evolve_equals_repeated_step_and_zero_iters():
    rng = np.random.default_rng(12)
    I = rng.uniform(0, 255, size=(6, 7, 8))
    phi = rng.normal(0, 2, size=I.shape)
    p = dict(PARAMS_PAPER3D, sigma=1.0)
    ref = phi
    for _ in range(3):
        ref = oracle.step(I, ref, p)
    np.testing.assert_array_equal(oracle.evolve(I, phi, p, 3), ref)
    np.testing.assert_array_equal(oracle.evolve(I, phi, p, 0), phi)


def test_openmp_build_is_bitwise_identical():
    rng = np.random.default_rng(13)
    I = rng.uniform(0, 255, size=(12, 13, 14))
    phi = rng.normal(0, 2, size=I.shape)
    a = oracle.evolve(I, phi, PARAMS_C1, 2, omp=False)
    b = oracle.evolve(I, phi, PARAMS_C1, 2, omp=True)
    np.testing.assert_array_equal(a, b)
