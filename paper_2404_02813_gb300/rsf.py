"""Python binding of librsf.so (include/rsf.h): argument marshalling only.

Every step of the level-set iteration runs in the library's CUDA kernels;
this module passes pointers, sizes and scalars through ctypes.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; volumes are [nz, ny, nx], x
fastest.  If the library has not been built, every call raises -- there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsf.so")

RSF_OK, RSF_PENDING, RSF_SUSPENDED = 0, 1, 2
STATUS_NAMES = {0: "RSF_OK", 1: "RSF_PENDING", 2: "RSF_SUSPENDED", -1: "RSF_E_INVAL", -2: "RSF_E_NOMEM", -3: "RSF_E_CUDA",
                -4: "RSF_E_TIMEOUT", -5: "RSF_E_NOTFOUND", -6: "RSF_E_BUSY", -7: "RSF_E_CANCELLED"}
RSF_U8, RSF_U16, RSF_F32 = 0, 1, 2
STAGES = ("f1", "f2", "g", "kappa", "lap")

EXPORTED = ("rsf_create", "rsf_destroy", "rsf_stream", "rsf_evolve", "rsf_step_stages", "rsf_prof_enable",
            "rsf_prof_count", "rsf_prof_name", "rsf_prof_get", "rsf_last_error", "rsf_evolve_noalloc",
            "rsf_set_option", "rsf_evolve_batch", "rsf_submit", "rsf_poll", "rsf_wait", "rsf_cancel",
            "rsf_serve_stats", "rsf_evolve_curtain", "rsf_init_phi0", "rsf_overlap", "rsf_isosurface",
            "rsf_suspend", "rsf_autotune_report")

OPT_PATH, OPT_ZCHUNK, OPT_STORAGE, OPT_AUTOTUNE, OPT_GRAPH, OPT_FAULT_ADMISSION, OPT_SERVE_SLOTS = 1, 2, 3, 4, 5, 6, 7
OPT_FORCE = 8
OPT_POISON = 9
OPT_FAULT_UPLOAD = 10
OPT_FAULT_WAIT = 11
PATHS = {"auto": 0, "passes": 1, "tiled": 2}
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
# data-term forms: Li et al.'s (default) and the paper's Eq. (15) with sigma_2 = 0
FORCES = {"li": 0, "eq15": 1}

NOALLOC_MAX_VOXELS = 1 << 18


class Brick(ctypes.Structure):
    """rsf_brick (include/rsf.h)."""
    _fields_ = [("volume", ctypes.c_void_p), ("vt", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("phi0", ctypes.c_void_p), ("phi_out", ctypes.c_void_p),
                ("sigma", ctypes.c_float), ("eps", ctypes.c_float), ("lambda1", ctypes.c_float),
                ("lambda2", ctypes.c_float), ("nu", ctypes.c_float), ("mu", ctypes.c_float), ("dt", ctypes.c_float),
                ("iters", ctypes.c_int32)]


class Request(ctypes.Structure):
    """rsf_request (include/rsf.h)."""
    _fields_ = Brick._fields_ + [("storage", ctypes.c_int32), ("halo", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class ServeStat(ctypes.Structure):
    """rsf_serve_stat (include/rsf.h)."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("voxel_iterations", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("latency_p50_s", ctypes.c_double), ("latency_p99_s", ctypes.c_double),
                ("latency_max_s", ctypes.c_double), ("suspended", ctypes.c_uint64)]


class RSFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librsf.so and declare its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librsf.so is not built ({path}); run __graft_entry__.build() first")
    L = ctypes.CDLL(path)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    L.rsf_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32]
    L.rsf_create.restype = i32
    L.rsf_destroy.argtypes = [vp]
    L.rsf_destroy.restype = None
    L.rsf_stream.argtypes = [vp]
    L.rsf_stream.restype = vp
    L.rsf_evolve.argtypes = [vp, vp, i32, i64, i64, i64, vp, vp, f32, f32, f32, f32, f32, f32, f32, i32]
    L.rsf_evolve.restype = i32
    L.rsf_step_stages.argtypes = [vp, vp, i32, i64, i64, i64, vp, vp, vp, f32, f32, f32, f32, f32, f32, f32]
    L.rsf_step_stages.restype = i32
    L.rsf_prof_enable.argtypes = [vp, i32]
    L.rsf_prof_enable.restype = i32
    L.rsf_prof_count.argtypes = []
    L.rsf_prof_count.restype = i32
    L.rsf_prof_name.argtypes = [i32]
    L.rsf_prof_name.restype = ctypes.c_char_p
    L.rsf_prof_get.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
    L.rsf_prof_get.restype = i32
    L.rsf_evolve_noalloc.argtypes = [vp, i32, i64, i64, i64, vp, vp, f32, f32, f32, f32, f32, f32, f32, i32, vp]
    L.rsf_evolve_noalloc.restype = i32
    L.rsf_autotune_report.argtypes = [vp, ctypes.c_char_p, i32]
    L.rsf_autotune_report.restype = i32
    L.rsf_evolve_batch.argtypes = [vp, ctypes.POINTER(Brick), i32]
    L.rsf_evolve_batch.restype = i32
    L.rsf_evolve_curtain.argtypes = [vp, vp, i32, i64, i64, i64, vp, vp, f32, f32, f32, f32, f32, f32, f32, i32, i32, i32]
    L.rsf_evolve_curtain.restype = i32
    L.rsf_init_phi0.argtypes = [vp, vp, i32, i64, i64, i64, f32, f32, f32, vp, ctypes.POINTER(i64), vp, vp]
    L.rsf_init_phi0.restype = i32
    L.rsf_overlap.argtypes = [vp, vp, vp, i64, ctypes.POINTER(i64)]
    L.rsf_overlap.restype = i32
    L.rsf_isosurface.argtypes = [vp, vp, i64, i64, i64, f32, vp, vp, i64, ctypes.POINTER(i64)]
    L.rsf_isosurface.restype = i32
    L.rsf_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.rsf_submit.restype = i32
    L.rsf_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    L.rsf_poll.restype = i32
    L.rsf_wait.argtypes = [vp, ctypes.c_uint64, i32]
    L.rsf_wait.restype = i32
    L.rsf_cancel.argtypes = [vp, ctypes.c_uint64]
    L.rsf_cancel.restype = i32
    L.rsf_suspend.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32)]
    L.rsf_suspend.restype = i32
    L.rsf_serve_stats.argtypes = [vp, ctypes.POINTER(ServeStat)]
    L.rsf_serve_stats.restype = i32
    L.rsf_set_option.argtypes = [vp, i32, i64]
    L.rsf_set_option.restype = i32
    L.rsf_last_error.argtypes = []
    L.rsf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int):
    if st < 0:
        raise RSFError(st, load_library().rsf_last_error().decode())
    return st


def _ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _order_after_caller(*arrays):
    """The library's stream follows the legacy default stream; work the caller
    queued on another torch stream is finished first."""
    if any(getattr(a, "is_cuda", False) for a in arrays):
        import torch
        cur = torch.cuda.current_stream()
        if cur != torch.cuda.default_stream():
            cur.synchronize()


def _vol_dtype(a) -> int:
    name = str(a.dtype).replace("torch.", "")
    if name == "uint8":
        return RSF_U8
    if name == "uint16":
        return RSF_U16
    if name == "float32":
        return RSF_F32
    raise TypeError(f"volume dtype must be uint8, uint16 or float32, not {name}")


def _shape(a):
    s = tuple(a.shape)
    if len(s) != 3:
        raise ValueError("expected a 3-D [nz, ny, nx] array")
    return s


@dataclass
class Params:
    """Scalars of the update (Eqs. 1, 6, 10-14)."""
    sigma: float = 3.0
    eps: float = 1.0
    lambda1: float = 1.0
    lambda2: float = 2.0
    nu: float = 0.004 * 255.0 ** 2
    mu: float = 1.0
    dt: float = 0.1

    @classmethod
    def of(cls, p) -> "Params":
        if isinstance(p, Params):
            return p
        return cls(**{k: float(p[k]) for k in ("sigma", "eps", "lambda1", "lambda2", "nu", "mu", "dt")})

    def tuple(self):
        return (self.sigma, self.eps, self.lambda1, self.lambda2, self.nu, self.mu, self.dt)


class Context:
    """One rsf_ctx: a device, an HBM budget and a CUDA stream."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        L = load_library()
        h = ctypes.c_void_p()
        _check(L.rsf_create(ctypes.byref(h), int(device), int(hbm_budget_bytes), 0))
        self._h = h
        self.device = int(device)
        self._live = {}  # ticket -> the submitted buffers, kept alive while the library uses them

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().rsf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def stream_handle(self) -> int:
        return int(load_library().rsf_stream(self._h) or 0)

    def evolve(self, volume, phi0, params, iters: int, out=None):
        """Run `iters` iterations from phi0; returns `out` (allocated like phi0 if None)."""
        p = Params.of(params)
        nz, ny, nx = _shape(volume)
        if _shape(phi0) != (nz, ny, nx):
            raise ValueError("volume and phi0 shapes differ")
        if str(phi0.dtype).replace("torch.", "") != "float32":
            raise TypeError("phi0 must be float32")
        if out is None:
            out = phi0.clone() if hasattr(phi0, "clone") else np.empty_like(phi0)
        _order_after_caller(volume, phi0, out)
        _check(load_library().rsf_evolve(self._h, _ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi0),
                                         _ptr(out), *p.tuple(), int(iters)))
        return out

    def evolve_curtain(self, volume, phi0, params, iters: int, edge: int, curtain: int, out=None):
        """rsf_evolve_curtain: overlapping sub-volumes of `edge` voxels evolved together and
        merged by linear interpolation across `curtain` voxels; returns `out`."""
        p = Params.of(params)
        nz, ny, nx = _shape(volume)
        if _shape(phi0) != (nz, ny, nx):
            raise ValueError("volume and phi0 shapes differ")
        if out is None:
            out = phi0.clone() if hasattr(phi0, "clone") else np.empty_like(phi0)
        _order_after_caller(volume, phi0, out)
        _check(load_library().rsf_evolve_curtain(self._h, _ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi0),
                                                 _ptr(out), *p.tuple(), int(iters), int(edge), int(curtain)))
        return out

    def init_phi0(self, volume, blob_sigma: float, rel_threshold: float, r0: float, seeds=None, response=None):
        """rsf_init_phi0: returns (phi0, number of seeds); `seeds` (uint8) and `response`
        (float32), shaped like the volume, receive the seed mask and the blob response."""
        nz, ny, nx = _shape(volume)
        if hasattr(volume, "new_empty"):
            phi0 = volume.new_empty((nz, ny, nx), dtype=__import__("torch").float32)
        else:
            phi0 = np.empty((nz, ny, nx), dtype=np.float32)
        count = ctypes.c_int64(0)
        _order_after_caller(volume, phi0)
        _check(load_library().rsf_init_phi0(self._h, _ptr(volume), _vol_dtype(volume), nx, ny, nz,
                                            float(blob_sigma), float(rel_threshold), float(r0), _ptr(phi0),
                                            ctypes.byref(count), _ptr(seeds) if seeds is not None else None,
                                            _ptr(response) if response is not None else None))
        return phi0, int(count.value)

    def overlap(self, phi, truth) -> dict:
        """rsf_overlap: counts of phi > 0, truth and both, with Dice and Jaccard."""
        n = 1
        for d in _shape(phi):
            n *= d
        if _shape(truth) != _shape(phi):
            raise ValueError("phi and truth shapes differ")
        c = (ctypes.c_int64 * 3)()
        _order_after_caller(phi, truth)
        _check(load_library().rsf_overlap(self._h, _ptr(phi), _ptr(truth), n, c))
        a, b, both = int(c[0]), int(c[1]), int(c[2])
        return {"segmented": a, "truth": b, "both": both,
                "dice": 2.0 * both / (a + b) if a + b else 1.0,
                "jaccard": both / (a + b - both) if a + b - both else 1.0}

    def isosurface(self, phi, iso: float = 0.0, with_keys: bool = True):
        """rsf_isosurface: (triangles [T, 3, 3] as x, y, z, keys [T]) as numpy arrays."""
        nz, ny, nx = _shape(phi)
        count = ctypes.c_int64(0)
        _order_after_caller(phi)
        L = load_library()
        _check(L.rsf_isosurface(self._h, _ptr(phi), nx, ny, nz, float(iso), None, None, 0, ctypes.byref(count)))
        cap = int(count.value)
        tri = np.empty((cap, 3, 3), dtype=np.float32)
        keys = np.empty(cap, dtype=np.int64) if with_keys else None
        if cap:
            _check(L.rsf_isosurface(self._h, _ptr(phi), nx, ny, nz, float(iso), tri.ctypes.data,
                                    keys.ctypes.data if with_keys else None, cap, ctypes.byref(count)))
        return tri, keys

    def step_stages(self, volume, phi, params, phi_next=None, stages=None):
        """One iteration with the stage fields; returns (phi_next, stages[5, nz, ny, nx])."""
        p = Params.of(params)
        nz, ny, nx = _shape(volume)
        if phi_next is None:
            phi_next = phi.clone() if hasattr(phi, "clone") else np.empty_like(phi)
        if stages is None:
            if hasattr(phi, "new_empty"):
                stages = phi.new_empty((len(STAGES), nz, ny, nx))
            else:
                stages = np.empty((len(STAGES), nz, ny, nx), dtype=np.float32)
        _order_after_caller(volume, phi, phi_next, stages)
        _check(load_library().rsf_step_stages(self._h, _ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi),
                                              _ptr(phi_next), _ptr(stages), *p.tuple()))
        return phi_next, stages

    def set_option(self, key: int, value: int):
        _check(load_library().rsf_set_option(self._h, int(key), int(value)))

    def set_path(self, name: str):
        """'auto' (tiled where instantiated, else passes), 'passes' or 'tiled'."""
        self.set_option(OPT_PATH, PATHS[name])

    def evolve_batch(self, items):
        """rsf_evolve_batch over (volume, phi0, params, iters[, out]) tuples; returns the outputs."""
        arr = (Brick * len(items))()
        outs, keep = [], []
        for k, it in enumerate(items):
            volume, phi0, params, iters = it[:4]
            out = it[4] if len(it) > 4 else (phi0.clone() if hasattr(phi0, "clone") else np.empty_like(phi0))
            p = Params.of(params)
            nz, ny, nx = _shape(volume)
            if _shape(phi0) != (nz, ny, nx) or _shape(out) != (nz, ny, nx):
                raise ValueError(f"brick {k}: shapes differ")
            arr[k] = Brick(_ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi0), _ptr(out), *p.tuple(), int(iters))
            outs.append(out)
            keep.append((volume, phi0))
        _order_after_caller(*[x for pair in keep for x in pair], *outs)
        _check(load_library().rsf_evolve_batch(self._h, arr, len(items)))
        return outs

    # serving -----------------------------------------------------------------
    def submit(self, volume, phi0, params, iters: int, out, storage: str = "f32", halo: int = -1, stream=None):
        """rsf_submit; returns the ticket.  `volume`, `phi0`, `out` stay owned by
        the caller and must stay valid until the ticket is no longer pending."""
        p = Params.of(params)
        nz, ny, nx = _shape(volume)
        if _shape(phi0) != (nz, ny, nx) or _shape(out) != (nz, ny, nx):
            raise ValueError("volume, phi0 and out shapes differ")
        _order_after_caller(volume, phi0, out)
        r = Request(_ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi0), _ptr(out), *p.tuple(), int(iters),
                    STORAGE[storage], int(halo), int(stream.cuda_stream) if stream is not None else 0)
        t = ctypes.c_uint64()
        _check(load_library().rsf_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._live[int(t.value)] = (volume, phi0, out)  # the library reads and writes them until the ticket resolves
        return int(t.value)

    def poll(self, ticket: int):
        """(status, latency_s): status RSF_PENDING (1), RSF_OK (0) or RSF_SUSPENDED (2); errors raise."""
        lat = ctypes.c_double(-1.0)
        try:
            st = _check(load_library().rsf_poll(self._h, int(ticket), ctypes.byref(lat)))
        except RSFError:
            self._live.pop(int(ticket), None)
            raise
        if st != 1:
            self._live.pop(int(ticket), None)
        return st, lat.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        try:
            st = _check(load_library().rsf_wait(self._h, int(ticket), int(timeout_ms)))
        except RSFError as e:
            if e.status != -4:  # not a timeout: the ticket is resolved
                self._live.pop(int(ticket), None)
            raise
        if st != 1:
            self._live.pop(int(ticket), None)
        return st

    def cancel(self, ticket: int):
        _check(load_library().rsf_cancel(self._h, int(ticket)))

    def suspend(self, ticket: int):
        """rsf_suspend: returns a ctypes.c_int32 that holds the completed iterations
        once the ticket resolves with SUSPENDED."""
        done = ctypes.c_int32(-1)
        _check(load_library().rsf_suspend(self._h, int(ticket), ctypes.byref(done)))
        # the library writes it when the ticket resolves: keep it alive until then
        self._live[int(ticket)] = tuple(self._live.get(int(ticket), ())) + (done,)
        return done

    def serve_stats(self) -> dict:
        st = ServeStat()
        _check(load_library().rsf_serve_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStat._fields_}

    def set_storage(self, name: str):
        """Storage of the intermediate fields: 'f32', 'bf16' or 'f16'."""
        self.set_option(OPT_STORAGE, STORAGE[name])

    def set_force(self, name: str):
        """Data-term form: 'li' (default) or 'eq15' (the paper's Eq. (15), sigma_2 = 0)."""
        self.set_option(OPT_FORCE, FORCES[name])

    # kernel timing ---------------------------------------------------------
    def autotune_report(self):
        """rsf_autotune_report parsed: one dict per tuned brick group."""
        buf = ctypes.create_string_buffer(1 << 16)
        _check(load_library().rsf_autotune_report(self._h, buf, len(buf)))
        out = []
        for line in buf.value.decode().splitlines():
            key, *fields = line.split()
            d = {"group": key}
            for f in fields:
                k, v = f.split("=", 1)
                d[k] = v if k == "order" else (float(v) if "ms" in k else int(v))
            out.append(d)
        return out

    def prof_enable(self, on: bool = True):
        _check(load_library().rsf_prof_enable(self._h, 1 if on else 0))

    def prof_get(self) -> Dict[str, tuple]:
        L = load_library()
        out = {}
        for k in range(L.rsf_prof_count()):
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            _check(L.rsf_prof_get(self._h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[L.rsf_prof_name(k).decode()] = (int(n.value), float(ms.value))
        return out


_default: Dict[int, Context] = {}


def context(device: int = 0) -> Context:
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def evolve(volume, phi0, sigma=3.0, eps=1.0, lambda1=1.0, lambda2=2.0, nu=0.004 * 255.0 ** 2, mu=1.0, dt=0.1,
           iters=50, out=None, device: Optional[int] = None):
    """rsf_evolve on the default context of `device` (the tensor's device, else 0)."""
    if device is None:
        device = volume.device.index if getattr(volume, "is_cuda", False) else 0
    p = Params(sigma, eps, lambda1, lambda2, nu, mu, dt)
    return context(device).evolve(volume, phi0, p, iters, out=out)


def evolve_noalloc(volume, phi0, params, iters: int, out, stream=None):
    """rsf_evolve_noalloc: the evolution for volumes of at most 262144 voxels
    without any device allocation, for callers that must not allocate GPU
    memory (their device memory belongs to a pool they do not control, or an
    allocation's implicit synchronisation is not acceptable).  `volume`,
    `phi0` and `out` must be CUDA tensors; the work is queued on `stream`
    (a torch.cuda.Stream, default the current stream) and is complete when that
    stream is.  Overlapping calls race on the library's shared static scratch.
    """
    import torch
    p = Params.of(params)
    nz, ny, nx = _shape(volume)
    if _shape(phi0) != (nz, ny, nx) or _shape(out) != (nz, ny, nx):
        raise ValueError("volume, phi0 and out shapes differ")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().rsf_evolve_noalloc(_ptr(volume), _vol_dtype(volume), nx, ny, nz, _ptr(phi0), _ptr(out),
                                             *p.tuple(), int(iters), int(s.cuda_stream)))
    return out
