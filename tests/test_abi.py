"""CPU-side checks of the C ABI: librsf.so builds, loads, exports every
function include/rsf.h declares, and reports errors without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rsf_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2404_02813_gb300 import build, rsf
    build.build()
    return rsf.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rsf_create", "rsf_destroy", "rsf_evolve", "rsf_last_error", "rsf_step_stages"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_2404_02813_gb300", "librsf.so"))
    missing = [n for n in sorted(_declared()) if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2404_02813_gb300 import rsf
    assert set(rsf.EXPORTED) >= _declared() - {"rsf_submit", "rsf_poll", "rsf_wait", "rsf_cancel"}


def test_null_context_is_invalid_argument(lib):
    st = lib.rsf_evolve(None, None, 0, 4, 4, 4, None, None, 3.0, 1.0, 1.0, 2.0, 1.0, 1.0, 0.1, 1)
    assert st == -1
    assert b"null context" in lib.rsf_last_error()


def test_create_reports_errors_without_aborting(lib):
    import torch
    h = ctypes.c_void_p()
    st = lib.rsf_create(ctypes.byref(h), 0, 0, 7)   # flags must be 0
    assert st == -1 and not h.value
    if not torch.cuda.is_available():
        st = lib.rsf_create(ctypes.byref(h), 0, 0, 0)
        assert st == -3 and not h.value
        assert len(lib.rsf_last_error()) > 0


def test_prof_names(lib):
    n = lib.rsf_prof_count()
    names = [lib.rsf_prof_name(k).decode() for k in range(n)]
    assert len(set(names)) == n and all(s.startswith("rsf_") for s in names)
    assert lib.rsf_prof_name(n) is None


def test_set_option_rejects_bad_keys_without_a_context(lib):
    assert lib.rsf_set_option(None, 1, 0) == -1


def test_serving_entry_points_validate_without_a_gpu(lib):
    import ctypes as C
    t = C.c_uint64()
    assert lib.rsf_submit(None, None, C.byref(t)) == -1
    assert lib.rsf_poll(None, 1, None) == -1
    assert lib.rsf_wait(None, 1, 0) == -1
    assert lib.rsf_cancel(None, 1) == -1
    assert lib.rsf_evolve_batch(None, None, 0) == -1


def test_new_entry_points_validate_without_a_gpu(lib):
    import ctypes as C
    n = C.c_int64()
    done = C.c_int32()
    assert lib.rsf_suspend(None, 1, C.byref(done)) == -1
    assert lib.rsf_isosurface(None, None, 4, 4, 4, C.c_float(0.0), None, None, 0, C.byref(n)) == -1
    assert lib.rsf_overlap(None, None, None, 0, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without librsf.so the binding raises instead of computing anything."""
    from paper_2404_02813_gb300 import rsf
    saved = rsf._lib
    rsf._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            rsf.load_library(str(tmp_path / "librsf.so"))
    finally:
        rsf._lib = saved


def test_binding_constants_match_the_header():
    """Every RSF_OPT_*, RSF_FORCE_*, RSF_PATH_* and status code the header
    defines has the same value in the binding (the binding passes them through)."""
    from paper_2404_02813_gb300 import rsf
    txt = open(os.path.join(ROOT, "include", "rsf.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(RSF_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt)}
    opts = {k[len("RSF_"):]: v for k, v in defs.items() if k.startswith("RSF_OPT_")}
    assert opts, "no options found in the header"
    for name, v in opts.items():
        assert getattr(rsf, name) == v, name
    for k, v in defs.items():
        if k.startswith("RSF_FORCE_"):
            assert rsf.FORCES[k[len("RSF_FORCE_"):].lower()] == v, k
        elif k.startswith("RSF_PATH_"):
            assert rsf.PATHS[k[len("RSF_PATH_"):].lower()] == v, k
    for k in ("RSF_OK", "RSF_E_INVAL", "RSF_E_NOMEM", "RSF_E_CUDA", "RSF_E_TIMEOUT", "RSF_E_CANCELLED"):
        assert k in defs, k
    assert defs["RSF_E_CUDA"] == -3 and defs["RSF_OPT_FAULT_WAIT"] == 11
