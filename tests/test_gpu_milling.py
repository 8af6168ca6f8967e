"""The 1024^3 uint8 milling-like workload with 16-bit (BF16, FP16) storage of
the intermediate fields, sigma = 3, the 64^3 parity configuration's RSF
parameters.

* A 128^3 sub-brick of the field, solved as its own volume, against the FP64
  oracle's full step, one iteration from the GPU's own states (the reduced-
  storage bound of test_gpu_reduced).
* The full 1024^3 volume in the benchmark's launch configuration: one
  iteration from the state after two, on sampled voxels against the oracle's
  direct-sum update, the storage allowance taken from the oracle's e1, e2 at
  each voxel.
* The full volume after the configuration's 300 iterations against FP32
  storage on the GPU: the segmentations (phi > 0) disagree no more than FP32
  disagrees with itself after a one-ulp random perturbation of phi0 (the
  iteration map's own sensitivity, see test_oracle_dynamics), with a margin.
"""
import numpy as np
import pytest

import oracle
from paper_2404_02813_gb300 import rsf, synth

from _parity import C0, FP32_EPS, assert_phi_close, storage_force_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = {"f16": 2e-2, "bf16": 2e-2}
UNIT = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
SIGN = {"f16": 1e-4, "bf16": 1e-4}
E = 1024


@pytest.fixture(scope="module")
def field():
    return synth.MillingField(extent_xyz=(E, E, E))


@pytest.fixture(scope="module")
def full(field):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol = synth.field_volume(field)
    return vol, synth.mean_rule_phi0(vol)


def _ctx(storage):
    c = rsf.Context(0)
    c.set_storage(storage)
    return c


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_milling_subbrick_per_iteration(field, storage):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    vol = field.box((448, 448, 448), (128, 128, 128))
    phi0 = synth.mean_rule_phi0(vol)
    p = synth.RSFParams().as_dict()
    ctx = _ctx(storage)
    try:
        v = torch.from_numpy(vol).cuda()
        for n in (0, 5):
            phi_n = ctx.evolve(v, torch.from_numpy(phi0).cuda(), p, n)
            nxt = ctx.evolve(v, phi_n, p, 1).cpu().numpy()
            phi_n = phi_n.cpu().numpy()
            ref, dump = oracle.step(vol.astype(np.float64), phi_n.astype(np.float64), p, dump=True, omp=True)
            force = storage_force_tol(phi_n, dump, p, UNIT[storage])
            err = assert_phi_close(nxt, ref, phi_n, rel=REL[storage], force=force, sign_max=SIGN[storage],
                                   what=f"milling 128^3 sub-brick {storage} step {n}")
            print(f"milling sub-brick {storage} step {n}: max |dphi| = {err:.3e}")
    finally:
        ctx.close()


def _samples(rng):
    pts = {(x, y, z) for x in (0, E - 1) for y in (0, E - 1) for z in (0, E - 1)}
    edges = (0, 1, 31, 32, 511, 512, 1016, 1023)
    for _ in range(24):
        pts.add(tuple(int(rng.choice(edges)) for _ in range(3)))
    while len(pts) < 64:
        pts.add(tuple(int(v) for v in rng.integers(0, E, size=3)))
    return sorted(pts)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_milling_fullsize_sampled_voxels(full, storage):
    vol, phi0 = full
    p = synth.RSFParams().as_dict()
    ctx = _ctx(storage)
    try:
        v = torch.from_numpy(vol).cuda()
        phi_n = ctx.evolve(v, torch.from_numpy(phi0).cuda(), p, 2)
        nxt = ctx.evolve(v, phi_n, p, 1).cpu().numpy()
        phi_n = phi_n.cpu().numpy()
        del v
    finally:
        ctx.close()
    I64 = vol.astype(np.float64)
    P64 = phi_n.astype(np.float64)
    worst = 0.0
    eps, dt = p["eps"], p["dt"]
    for (x, y, z) in _samples(np.random.default_rng(1024)):
        ref, t = oracle.point_next(I64, P64, p, x, y, z, terms=True)
        ph = P64[z, y, x]
        delta = (eps / np.pi) / (eps * eps + ph * ph)
        force = 4.0 * UNIT[storage] * dt * delta * (p["lambda1"] * abs(t["e1"]) + p["lambda2"] * abs(t["e2"]))
        tol = REL[storage] * C0 + 8.0 * FP32_EPS * max(abs(ph), abs(ref)) + force
        got = float(nxt[z, y, x])
        assert abs(got - ref) <= tol, f"{storage} voxel {(x, y, z)}: gpu {got!r} oracle {ref!r} tol {tol:.3e}"
        worst = max(worst, abs(got - ref) / tol)
    print(f"milling 1024^3 {storage}: worst |d|/tol = {worst:.3f} over 64 sampled voxels")


def test_milling_fullsize_reduced_against_fp32(full):
    vol, phi0 = full
    p = synth.RSFParams().as_dict()
    iters = 300
    rng = np.random.default_rng(77)
    phi0_pert = np.nextafter(phi0, np.where(rng.random(phi0.shape) < 0.5, -np.inf, np.inf).astype(np.float32))
    runs = {"f32": ("f32", phi0), "f32_perturbed": ("f32", phi0_pert), "f16": ("f16", phi0), "bf16": ("bf16", phi0)}
    res = {}
    for name, (storage, ph) in runs.items():
        ctx = _ctx(storage)
        try:
            out = ctx.evolve(torch.from_numpy(vol).cuda(), torch.from_numpy(ph).cuda(), p, iters)
            res[name] = (out > 0).cpu().numpy()
            del out
        finally:
            ctx.close()
    ref = res["f32"]

    def compare(a):
        dis = float(np.mean(a != ref))
        dice = 2.0 * np.logical_and(a, ref).sum() / max(int(a.sum()) + int(ref.sum()), 1)
        return dis, dice

    env, env_dice = compare(res["f32_perturbed"])
    print(f"milling 1024^3 after {iters} iterations, FP32 vs FP32 from a one-ulp perturbed phi0: "
          f"sign disagreement {env:.3e}, Dice {env_dice:.5f}")
    for storage in ("f16", "bf16"):
        dis, dice = compare(res[storage])
        print(f"milling 1024^3 after {iters} iterations, {storage} vs f32: sign disagreement {dis:.3e}, Dice {dice:.5f}")
        assert dis <= max(1.5 * env, 1e-4), f"{storage}: disagreement {dis} against the FP32 envelope {env}"
        assert dice >= 0.98, f"{storage}: Dice {dice}"
