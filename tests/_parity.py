"""Shared helpers of the GPU parity tests (tolerances, array transfer, inputs)."""
import numpy as np

C0 = 2.0
FP32_EPS = 2.0 ** -23


def phi_tol(phi_n, phi_ref, rel=1e-3, force=None):
    """Per-voxel bound on |phi_gpu - phi_oracle| after one iteration from phi_n.

    ``rel * c0`` absolute (1e-3 for the FP32 path, 2e-2 for 16-bit storage), plus
    eight FP32 ulps of the magnitude of phi involved: phi is stored in FP32, so
    its rounding alone is half an ulp of |phi|, and the update adds terms of that
    size (phi reaches ~1e5 on 16-bit data after one step).  With 16-bit storage
    of intermediate fields, ``force`` is the extra per-voxel allowance for the
    storage rounding that enters the data terms (see ``storage_force_tol``).
    """
    phi_n = np.asarray(phi_n, dtype=np.float64)
    mag = np.maximum(np.abs(phi_n), np.abs(phi_ref))
    tol = rel * C0 + 8.0 * FP32_EPS * mag
    return tol if force is None else tol + force


def storage_force_tol(phi_n, dump, params, unit_roundoff, factor=4.0):
    """Allowance for 16-bit storage of the fits: the data terms e1, e2 are formed
    from stored fields rounded to ``unit_roundoff`` relative to their own size, and
    enter the step as dt * delta(phi_n) * (lambda1 e1 - lambda2 e2); the bound is
    ``factor`` roundoffs of the non-cancelled magnitude dt*delta*(l1|e1| + l2|e2|)."""
    phi_n = np.asarray(phi_n, dtype=np.float64)
    eps = params["eps"]
    delta = (eps / np.pi) / (eps * eps + phi_n * phi_n)
    mag = params["lambda1"] * np.abs(dump["e1"]) + params["lambda2"] * np.abs(dump["e2"])
    return factor * unit_roundoff * params["dt"] * delta * mag


def assert_phi_close(out, ref, phi_n, rel=1e-3, what="", force=None, sign_max=1e-4):
    out = np.asarray(out, dtype=np.float64)
    err = np.abs(out - ref)
    tol = phi_tol(phi_n, ref, rel, force)
    bad = err > tol
    assert np.all(np.isfinite(out)), f"{what}: non-finite values in the GPU result"
    if bad.any():
        i = np.unravel_index(np.argmax(err - tol), err.shape)
        raise AssertionError(f"{what}: {bad.sum()} voxels over tolerance; worst at {i}: gpu {out[i]!r} "
                             f"oracle {ref[i]!r} |d| {err[i]:.3e} tol {tol[i]:.3e} (max |d| {err.max():.3e})")
    sign = np.mean(np.sign(out) != np.sign(ref))
    assert sign <= sign_max, f"{what}: sign disagreement {sign:.2e}"
    return float(err.max())


def paper_c1():
    """The 64^3 uint8 vessel-tree workload with its parameters and box phi0."""
    from paper_2404_02813_gb300 import synth
    vol = synth.tree_volume_u8()
    phi0 = synth.box_phi0(vol.shape, 32)
    return vol, phi0, synth.RSFParams().as_dict()
