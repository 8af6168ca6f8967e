"""rsf_evolve_noalloc through the C ABI against rsf_evolve.

rsf_evolve_noalloc serves callers that must not allocate GPU memory while they
run (their device memory belongs to a pool they do not control, or the
synchronisation an allocation can cause is not acceptable); it keeps its
working fields in a static array built into the library.  These tests check
that two calls in a row -- the second one finding the first one's leftovers in
that shared array -- each give the same result as the allocating entry point,
within the per-voxel tolerance the other GPU tests use, and that volumes above
its static limit are refused.  This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2404_02813_gb300 import rsf, synth

from _parity import phi_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = rsf.Context(0)
    c.set_path("passes")   # the schedule rsf_evolve_noalloc runs
    yield c
    c.close()


def _case(shape, seed, iters):
    vol = synth.tree_volume_u8(shape, brick=seed, n_segments=12)
    phi0 = synth.box_phi0(shape, min(shape) // 2)
    return vol, phi0, synth.RSFParams().as_dict(), iters


def test_noalloc_matches_evolve_on_two_calls_in_a_row(ctx):
    # the second call is smaller and ragged, so stale contents of the shared
    # static array from the first call would show up in its result
    for shape, seed, iters in [((40, 44, 48), 1, 6), ((29, 31, 37), 2, 5)]:
        vol, phi0, p, iters = _case(shape, seed, iters)
        v = torch.from_numpy(vol).cuda()
        ph = torch.from_numpy(phi0).cuda()
        ref = ctx.evolve(v, ph, p, iters).cpu().numpy()
        out = torch.full_like(ph, float("nan"))
        s = torch.cuda.current_stream()
        rsf.evolve_noalloc(v, ph, p, iters, out, stream=s)
        s.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.abs(got.astype(np.float64) - ref)
        assert np.all(err <= phi_tol(ref, ref.astype(np.float64))), float(err.max())


def test_noalloc_output_may_alias_input(ctx):
    vol, phi0, p, iters = _case((24, 20, 28), 3, 3)
    v = torch.from_numpy(vol).cuda()
    ref = ctx.evolve(v, torch.from_numpy(phi0).cuda(), p, iters).cpu().numpy()
    ph = torch.from_numpy(phi0).cuda()
    rsf.evolve_noalloc(v, ph, p, iters, ph)
    torch.cuda.current_stream().synchronize()
    err = np.abs(ph.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= phi_tol(ref, ref.astype(np.float64)))


def test_noalloc_rejects_volumes_above_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    shape = (64, 64, 65)  # 266240 > 262144 voxels
    v = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    ph = torch.zeros(shape, dtype=torch.float32, device="cuda")
    with pytest.raises(rsf.RSFError) as e:
        rsf.evolve_noalloc(v, ph, synth.RSFParams().as_dict(), 1, ph)
    assert e.value.status == -1 and "limit" in str(e.value)
    with pytest.raises(rsf.RSFError) as e:   # host buffers are refused too
        rsf.evolve_noalloc(v.cpu()[:8, :8, :8].contiguous(), ph.cpu()[:8, :8, :8].contiguous(),
                           synth.RSFParams().as_dict(), 1, ph.cpu()[:8, :8, :8].contiguous())
    assert e.value.status == -1


def test_noalloc_rejects_memory_of_another_device():
    """Device memory of a GPU other than the current one is refused before any
    launch (without peer access a kernel would fault on it)."""
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    shape = (8, 8, 8)
    v = torch.zeros(shape, dtype=torch.uint8, device="cuda:1")
    ph = torch.zeros(shape, dtype=torch.float32, device="cuda:1")
    with torch.cuda.device(0):
        with pytest.raises(rsf.RSFError) as e:
            rsf.evolve_noalloc(v, ph, synth.RSFParams().as_dict(), 1, ph, stream=torch.cuda.current_stream(0))
    assert e.value.status == -1
