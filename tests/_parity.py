"""Shared helpers of the GPU parity tests (tolerances, array transfer, inputs)."""
import numpy as np

C0 = 2.0
FP32_EPS = 2.0 ** -23


def phi_tol(phi_n, phi_ref, rel=1e-3):
    """Per-voxel bound on |phi_gpu - phi_oracle| after one iteration from phi_n.

    ``rel * c0`` absolute (1e-3 for the FP32 path, 2e-2 for 16-bit storage), plus
    eight FP32 ulps of the magnitude of phi involved: phi is stored in FP32, so
    its rounding alone is half an ulp of |phi|, and the update adds terms of that
    size (phi reaches ~1e5 on 16-bit data after one step).
    """
    mag = np.maximum(np.abs(np.asarray(phi_n, dtype=np.float64)), np.abs(phi_ref))
    return rel * C0 + 8.0 * FP32_EPS * mag


def assert_phi_close(out, ref, phi_n, rel=1e-3, what=""):
    out = np.asarray(out, dtype=np.float64)
    err = np.abs(out - ref)
    tol = phi_tol(phi_n, ref, rel)
    bad = err > tol
    assert np.all(np.isfinite(out)), f"{what}: non-finite values in the GPU result"
    if bad.any():
        i = np.unravel_index(np.argmax(err - tol), err.shape)
        raise AssertionError(f"{what}: {bad.sum()} voxels over tolerance; worst at {i}: gpu {out[i]!r} "
                             f"oracle {ref[i]!r} |d| {err[i]:.3e} tol {tol[i]:.3e} (max |d| {err.max():.3e})")
    sign = np.mean(np.sign(out) != np.sign(ref))
    assert sign <= 1e-4, f"{what}: sign disagreement {sign:.2e}"
    return float(err.max())


def paper_c1():
    """The 64^3 uint8 vessel-tree workload with its parameters and box phi0."""
    from paper_2404_02813_gb300 import synth
    vol = synth.tree_volume_u8()
    phi0 = synth.box_phi0(vol.shape, 32)
    return vol, phi0, synth.RSFParams().as_dict()
