"""Thin ctypes binding of the C ABI in ``include/mbo.h`` and ``include/mbo_surface.h``.

Every function keeps the C name and only marshals arguments: tensors become
device (or, for the run loop, host) pointers, streams become ``cudaStream_t``
handles, and outputs are unpacked into Python values.  All arithmetic runs in
the CUDA library; there is no CPU fallback, and importing a function whose
library is missing raises.

Fields are ``torch.Tensor`` objects of shape ``(n*n, *dims)`` (channel
``i*n+j`` = matrix entry ``(i, j)``), contiguous, ``float32`` or ``float64``
matching the handle's dtype, on the handle's CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MBO_F32 = 1
MBO_F64 = 2
MBO_STEP_CONTINUE = 1

STATUS = {0: "MBO_OK", 1: "MBO_ERR_INVALID_ARG", 2: "MBO_ERR_UNSUPPORTED_SIZE", 3: "MBO_ERR_OOM",
          4: "MBO_ERR_CUDA", 5: "MBO_ERR_NUMERIC", 6: "MBO_ERR_DEVICE_TIMEOUT"}

EXPORTS = ("mbo_default_config", "mbo_create", "mbo_destroy", "mbo_diffuse", "mbo_project",
           "mbo_step", "mbo_lyapunov", "mbo_run_until_stationary", "mbo_profile_enable",
           "mbo_profile_read", "mbo_diffuse_noalloc", "mbo_step_volume", "mbo_run_volume",
           "mbo_batch_create", "mbo_batch_destroy",
           "mbo_batch_step", "mbo_batch_run", "mbo_batch_workspace_bytes", "mbo_batch_last_error",
           "mbo_workspace_bytes", "mbo_status_string", "mbo_last_error", "mbo_measure_fma_peaks",
           "mbo_selftest_wait_timeout", "mbo_launch_config")

SURFACE_EXPORTS = ("mbo_surface_band_width", "mbo_surface_heat_modes", "mbo_surface_sphere_band",
                   "mbo_surface_peanut_band",
                   "mbo_surface_create", "mbo_surface_destroy", "mbo_surface_get_params",
                   "mbo_surface_diffuse", "mbo_surface_step", "mbo_surface_step_volume",
                   "mbo_surface_profile_enable",
                   "mbo_surface_profile_read", "mbo_surface_workspace_bytes",
                   "mbo_surface_last_error")

SURFACE_PASSES = ("spread", "grid_fft", "interp", "project")

MBO_NOALLOC_SCRATCH_BYTES = 64 << 20

PASSES = ("row_fwd", "axis_fwd", "axis_fgi", "axis_inv", "axis_energy", "row_project", "row_inv",
          "project")


class MboError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mbo_config(C.Structure):
    _fields_ = [("fallback_sigma", C.c_double), ("check_interval", C.c_int), ("use_graph", C.c_int),
                ("row_threads", C.c_int), ("axis_threads", C.c_int), ("axis_tx", C.c_int),
                ("axis_stages", C.c_int), ("autotune", C.c_int), ("pdl", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class mbo_surface_params(C.Structure):
    _fields_ = [("h", C.c_double), ("M", C.c_int), ("nf", C.c_int), ("width", C.c_int),
                ("beta", C.c_double), ("R", C.c_double), ("center", C.c_double * 3),
                ("bins", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["center"] = tuple(self.center)
        return d


class mbo_stats(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_delta", C.c_double), ("det_flips", C.c_int64),
                ("fallback_points", C.c_int64), ("nonfinite", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; build it with "
                          "paper_1711_01365_gb300.build.build() (nvcc, sm_103a)")
    L = C.CDLL(path)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    L.mbo_default_config.argtypes = [C.POINTER(mbo_config)]
    L.mbo_default_config.restype = None
    L.mbo_create.argtypes = [C.POINTER(vp), C.c_int, i64p, C.c_int, C.c_double, C.c_int,
                             C.POINTER(mbo_config)]
    L.mbo_destroy.argtypes = [vp]
    L.mbo_diffuse.argtypes = [vp, vp, vp, vp]
    L.mbo_project.argtypes = [vp, vp, vp, vp, vp]
    L.mbo_step.argtypes = [vp, vp, C.c_int, C.POINTER(mbo_stats), vp]
    L.mbo_lyapunov.argtypes = [vp, vp, C.POINTER(C.c_double), vp]
    L.mbo_run_until_stationary.argtypes = [vp, vp, C.c_int, C.c_double, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), i64p, C.POINTER(mbo_stats), vp]
    L.mbo_profile_enable.argtypes = [vp, C.c_int]
    L.mbo_profile_read.argtypes = [vp, C.POINTER(C.c_double), i64p, C.c_int]
    L.mbo_diffuse_noalloc.argtypes = [C.c_int, i64p, C.c_int, C.c_double, C.c_int, vp, vp, vp]
    L.mbo_measure_fma_peaks.argtypes = [C.POINTER(C.c_double)] * 3
    L.mbo_selftest_wait_timeout.argtypes = [vp, C.c_int64, vp]
    L.mbo_launch_config.argtypes = [vp, C.POINTER(mbo_config)]
    L.mbo_step_volume.argtypes = [vp, vp, C.c_int64, C.POINTER(mbo_stats), vp]
    L.mbo_run_volume.argtypes = [vp, vp, C.c_int64, C.c_int, C.c_double, C.POINTER(C.c_int),
                                 C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.mbo_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), i64p,
                                   C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int,
                                   C.POINTER(mbo_config)]
    L.mbo_batch_destroy.argtypes = [vp]
    L.mbo_batch_step.argtypes = [vp, C.POINTER(vp), C.c_int, C.POINTER(mbo_stats), vp]
    L.mbo_batch_run.argtypes = [vp, C.POINTER(vp), C.c_int, C.c_double, C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(mbo_stats), vp]
    L.mbo_batch_workspace_bytes.argtypes = [vp]
    L.mbo_batch_workspace_bytes.restype = C.c_int64
    L.mbo_batch_last_error.argtypes = [vp]
    L.mbo_batch_last_error.restype = C.c_char_p
    L.mbo_workspace_bytes.argtypes = [vp]
    L.mbo_workspace_bytes.restype = C.c_int64
    L.mbo_status_string.argtypes = [C.c_int]
    L.mbo_status_string.restype = C.c_char_p
    L.mbo_last_error.argtypes = [vp]
    L.mbo_last_error.restype = C.c_char_p
    dp = C.POINTER(C.c_double)
    L.mbo_surface_band_width.argtypes = [C.c_double, C.c_double]
    L.mbo_surface_band_width.restype = C.c_double
    L.mbo_surface_heat_modes.argtypes = [C.c_double, C.c_double, C.c_double, dp, C.POINTER(C.c_int)]
    L.mbo_surface_sphere_band.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, vp, vp, vp,
                                          C.c_int64, i64p]
    L.mbo_surface_peanut_band.argtypes = [C.c_double, C.c_double, C.c_int, vp, vp, vp, C.c_int64, i64p]
    L.mbo_surface_create.argtypes = [C.POINTER(vp), C.c_int64, vp, vp, vp, C.c_int, C.c_double,
                                     C.c_double, C.c_int]
    L.mbo_surface_destroy.argtypes = [vp]
    L.mbo_surface_get_params.argtypes = [vp, C.POINTER(mbo_surface_params)]
    L.mbo_surface_diffuse.argtypes = [vp, vp, vp, vp]
    L.mbo_surface_step.argtypes = [vp, vp, C.POINTER(mbo_stats), vp]
    L.mbo_surface_step_volume.argtypes = [vp, vp, C.c_double, C.POINTER(mbo_stats), vp]
    L.mbo_surface_profile_enable.argtypes = [vp, C.c_int]
    L.mbo_surface_profile_read.argtypes = [vp, C.POINTER(C.c_double), i64p, C.c_int]
    L.mbo_surface_workspace_bytes.argtypes = [vp]
    L.mbo_surface_workspace_bytes.restype = C.c_int64
    L.mbo_surface_last_error.argtypes = [vp]
    L.mbo_surface_last_error.restype = C.c_char_p
    for f in ("mbo_surface_heat_modes", "mbo_surface_sphere_band", "mbo_surface_peanut_band", "mbo_surface_create",
              "mbo_surface_destroy", "mbo_surface_get_params", "mbo_surface_diffuse",
              "mbo_surface_step", "mbo_surface_step_volume", "mbo_surface_profile_enable",
              "mbo_surface_profile_read"):
        getattr(L, f).restype = C.c_int
    for f in ("mbo_create", "mbo_destroy", "mbo_diffuse", "mbo_project", "mbo_step", "mbo_lyapunov",
              "mbo_run_until_stationary", "mbo_profile_enable", "mbo_profile_read",
              "mbo_diffuse_noalloc", "mbo_step_volume", "mbo_run_volume", "mbo_batch_create",
              "mbo_batch_destroy", "mbo_batch_step",
              "mbo_batch_run"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(rc: int, h=None) -> None:
    if rc != 0:
        msg = lib().mbo_status_string(rc).decode()
        if h is not None:
            detail = lib().mbo_last_error(h).decode()
            if detail:
                msg += f" ({detail})"
        raise MboError(rc, msg)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def mbo_default_config() -> mbo_config:
    cfg = mbo_config()
    lib().mbo_default_config(C.byref(cfg))
    return cfg


def mbo_create(dims, n: int, tau: float, dtype: int = MBO_F32, cfg: mbo_config | None = None):
    """Create a handle for a field of the given dims ((Ny, Nx) or (Nz, Ny, Nx))."""
    h = C.c_void_p()
    d = (C.c_int64 * len(dims))(*[int(v) for v in dims])
    rc = lib().mbo_create(C.byref(h), len(dims), d, int(n), float(tau), int(dtype),
                          C.byref(cfg) if cfg is not None else None)
    _check(rc)
    return h


def mbo_destroy(h) -> None:
    _check(lib().mbo_destroy(h))


def mbo_diffuse(h, A, A_tilde, stream=None) -> None:
    _check(lib().mbo_diffuse(h, _ptr(A), _ptr(A_tilde), _stream(stream)), h)


def mbo_project(h, A_tilde, B, det_sign=None, stream=None) -> None:
    _check(lib().mbo_project(h, _ptr(A_tilde), _ptr(B), _ptr(det_sign), _stream(stream)), h)


def mbo_step(h, A, flags: int = 0, want_stats: bool = False, stream=None):
    st = mbo_stats()
    _check(lib().mbo_step(h, _ptr(A), int(flags), C.byref(st) if want_stats else None,
                          _stream(stream)), h)
    return st.as_dict() if want_stats else None


def mbo_lyapunov(h, A, stream=None) -> float:
    e = C.c_double(0.0)
    _check(lib().mbo_lyapunov(h, _ptr(A), C.byref(e), _stream(stream)), h)
    return e.value


def mbo_run_until_stationary(h, A, max_steps: int, tol: float, stream=None) -> dict:
    """Iterate in place; A may be a device tensor or a host array/tensor."""
    steps = C.c_int(0)
    stat = C.c_int(0)
    en = np.zeros(max_steps + 1, dtype=np.float64)
    md = np.zeros(max(max_steps, 1), dtype=np.float64)
    fl = np.zeros(max(max_steps, 1), dtype=np.int64)
    last = mbo_stats()
    rc = lib().mbo_run_until_stationary(
        h, _ptr(A), int(max_steps), float(tol), C.byref(steps), C.byref(stat),
        en.ctypes.data_as(C.POINTER(C.c_double)), md.ctypes.data_as(C.POINTER(C.c_double)),
        fl.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(last), _stream(stream))
    _check(rc, h)
    s = steps.value
    return {"steps": s, "stationary": bool(stat.value), "energies": en[: s + 1],
            "max_deltas": md[:s], "det_flips": fl[:s], "last": last.as_dict()}


def mbo_diffuse_noalloc(dims, n: int, tau: float, dtype: int, A, A_tilde, stream=None) -> None:
    """mbo_diffuse without a handle and without device allocation (scratch in a
    static 64 MiB device array inside the library; see include/mbo.h).

    With no handle to hold the sizes, tensor arguments are checked here: each
    must be contiguous, hold n*n*prod(dims) values of the dtype's type and sit
    on a CUDA device; ValueError otherwise (the kernels would read or write
    past a smaller buffer)."""
    want = int(n) * int(n) * int(np.prod([int(v) for v in dims]))
    for name, t in (("A", A), ("A_tilde", A_tilde)):
        if hasattr(t, "data_ptr") and hasattr(t, "numel"):
            import torch
            tdt = torch.float32 if int(dtype) == MBO_F32 else torch.float64
            if t.numel() != want:
                raise ValueError(f"{name} holds {t.numel()} values, the problem needs {want}")
            if t.dtype != tdt:
                raise ValueError(f"{name} is {t.dtype}, the call's dtype is {tdt}")
            if not t.is_contiguous():
                raise ValueError(f"{name} is not contiguous")
            if not t.is_cuda:
                raise ValueError(f"{name} is not on a CUDA device")
    d = (C.c_int64 * len(dims))(*[int(v) for v in dims])
    _check(lib().mbo_diffuse_noalloc(len(dims), d, int(n), float(tau), int(dtype), _ptr(A),
                                     _ptr(A_tilde), _stream(stream)))


def mbo_launch_config(h) -> dict:
    """The launch shapes the handle uses (after any autotuning)."""
    c = mbo_config()
    _check(lib().mbo_launch_config(h, C.byref(c)), h)
    return c.as_dict()


def mbo_selftest_wait_timeout(h, limit_cycles: int = 2_000_000, stream=None) -> int:
    """Run the bounded-wait timeout path on purpose (see include/mbo.h); returns
    the status code (MBO_ERR_DEVICE_TIMEOUT = 6 when the path works)."""
    return int(lib().mbo_selftest_wait_timeout(h, int(limit_cycles), _stream(stream)))


def mbo_measure_fma_peaks() -> dict:
    """SIMT multiply-add throughput of the current device in TFLOP/s:
    {"fp32": scalar FFMA, "fp32x2": packed pairs, "fp64": DFMA}."""
    a, b, c = C.c_double(0), C.c_double(0), C.c_double(0)
    _check(lib().mbo_measure_fma_peaks(C.byref(a), C.byref(b), C.byref(c)))
    return {"fp32": a.value, "fp32x2": b.value, "fp64": c.value}


def mbo_step_volume(h, A, n_plus: int = -1, want_stats: bool = False, stream=None):
    st = mbo_stats()
    _check(lib().mbo_step_volume(h, _ptr(A), int(n_plus), C.byref(st) if want_stats else None,
                                 _stream(stream)), h)
    return st.as_dict() if want_stats else None


def mbo_run_volume(h, A, n_plus: int, max_steps: int, tol: float, stream=None) -> dict:
    steps = C.c_int(0)
    stat = C.c_int(0)
    en = np.zeros(max_steps + 1, dtype=np.float64)
    _check(lib().mbo_run_volume(h, _ptr(A), int(n_plus), int(max_steps), float(tol), C.byref(steps),
                                C.byref(stat), en.ctypes.data_as(C.POINTER(C.c_double)),
                                _stream(stream)), h)
    s = steps.value
    return {"steps": s, "stationary": bool(stat.value), "energies": en[: s + 1]}


def mbo_profile_enable(h, enable: bool = True) -> None:
    _check(lib().mbo_profile_enable(h, 1 if enable else 0), h)


def mbo_profile_read(h) -> dict:
    """{pass name: (total ms, launches)} since the last mbo_profile_enable."""
    n = len(PASSES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(lib().mbo_profile_read(h, ms, cnt, n), h)
    return {PASSES[i]: (ms[i], cnt[i]) for i in range(n)}


def _bcheck(rc: int, b) -> None:
    if rc != 0:
        msg = lib().mbo_status_string(rc).decode()
        if b is not None:
            d = lib().mbo_batch_last_error(b).decode()
            if d:
                msg += f" ({d})"
        raise MboError(rc, msg)


def mbo_batch_create(dims_list, n_list, tau_list, dtype: int = MBO_F32,
                     cfg: mbo_config | None = None):
    """Handle for a batch of independent fields (dims may differ per field)."""
    cnt = len(dims_list)
    nd = (C.c_int * cnt)(*[len(d) for d in dims_list])
    flat = []
    for d in dims_list:
        flat += [int(v) for v in d] + [0] * (3 - len(d))
    dd = (C.c_int64 * (3 * cnt))(*flat)
    nn = (C.c_int * cnt)(*[int(v) for v in n_list])
    tt = (C.c_double * cnt)(*[float(v) for v in tau_list])
    b = C.c_void_p()
    rc = lib().mbo_batch_create(C.byref(b), cnt, nd, dd, nn, tt, int(dtype),
                                C.byref(cfg) if cfg is not None else None)
    _bcheck(rc, None)
    return b


def mbo_batch_destroy(b) -> None:
    _bcheck(lib().mbo_batch_destroy(b), None)


def _ptrs(fields):
    return (C.c_void_p * len(fields))(*[_ptr(f) for f in fields])


def mbo_batch_step(b, fields, flags: int = 0, want_stats: bool = False, stream=None):
    st = (mbo_stats * len(fields))()
    _bcheck(lib().mbo_batch_step(b, _ptrs(fields), int(flags), st if want_stats else None,
                                 _stream(stream)), b)
    return [s.as_dict() for s in st] if want_stats else None


def mbo_batch_run(b, fields, max_steps: int, tol: float, stream=None) -> dict:
    cnt = len(fields)
    steps = (C.c_int * cnt)()
    stat = (C.c_int * cnt)()
    en = np.zeros((cnt, max_steps + 1), dtype=np.float64)
    last = (mbo_stats * cnt)()
    _bcheck(lib().mbo_batch_run(b, _ptrs(fields), int(max_steps), float(tol), steps, stat,
                                en.ctypes.data_as(C.POINTER(C.c_double)), last, _stream(stream)), b)
    return {"steps": list(steps), "stationary": [bool(x) for x in stat],
            "energies": [en[i, : steps[i] + 1] for i in range(cnt)],
            "last": [s.as_dict() for s in last]}


def mbo_batch_workspace_bytes(b) -> int:
    return int(lib().mbo_batch_workspace_bytes(b))


class Batch:
    """Owning wrapper of a batch handle."""

    def __init__(self, dims_list, n_list, tau_list, dtype: str = "f32", **cfg):
        c = mbo_default_config()
        for k, v in cfg.items():
            setattr(c, k, v)
        self.count = len(dims_list)
        self.b = mbo_batch_create(dims_list, n_list, tau_list,
                                  {"f32": MBO_F32, "f64": MBO_F64}[dtype], c)

    def close(self) -> None:
        if getattr(self, "b", None) is not None:
            mbo_batch_destroy(self.b)
            self.b = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def step(self, fields, flags=0, want_stats=False, stream=None):
        return mbo_batch_step(self.b, fields, flags, want_stats, stream)

    def run(self, fields, max_steps: int, tol: float, stream=None) -> dict:
        return mbo_batch_run(self.b, fields, max_steps, tol, stream)


def mbo_workspace_bytes(h) -> int:
    return int(lib().mbo_workspace_bytes(h))


def mbo_status_string(status: int) -> str:
    return lib().mbo_status_string(int(status)).decode()


def mbo_last_error(h) -> str:
    return lib().mbo_last_error(h).decode()


class Mbo:
    """Owning wrapper of a handle (closes it on ``close()`` / garbage collection)."""

    def __init__(self, dims, n: int, tau: float, dtype: str = "f32", **cfg):
        c = mbo_default_config()
        for k, v in cfg.items():
            setattr(c, k, v)
        self.dims, self.n, self.tau = tuple(int(d) for d in dims), int(n), float(tau)
        self.dtype = {"f32": MBO_F32, "f64": MBO_F64}[dtype]
        self.h = mbo_create(self.dims, self.n, self.tau, self.dtype, c)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            mbo_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def diffuse(self, A, out, stream=None):
        mbo_diffuse(self.h, A, out, stream)
        return out

    def project(self, At, out, det_sign=None, stream=None):
        mbo_project(self.h, At, out, det_sign, stream)
        return out

    def step(self, A, flags=0, want_stats=False, stream=None):
        return mbo_step(self.h, A, flags, want_stats, stream)

    def lyapunov(self, A, stream=None) -> float:
        return mbo_lyapunov(self.h, A, stream)

    def run(self, A, max_steps: int, tol: float, stream=None) -> dict:
        return mbo_run_until_stationary(self.h, A, max_steps, tol, stream)

    def step_volume(self, A, n_plus: int = -1, want_stats=False, stream=None):
        return mbo_step_volume(self.h, A, n_plus, want_stats, stream)

    def run_volume(self, A, n_plus: int, max_steps: int, tol: float, stream=None) -> dict:
        return mbo_run_volume(self.h, A, n_plus, max_steps, tol, stream)


# ---------------------------------------------------------------------------
# closed surfaces (include/mbo_surface.h)
# ---------------------------------------------------------------------------

def _scheck(rc: int, s=None) -> None:
    if rc != 0:
        msg = lib().mbo_status_string(rc).decode()
        if s is not None:
            detail = lib().mbo_surface_last_error(s).decode()
            if detail:
                msg += f" ({detail})"
        raise MboError(rc, msg)


def mbo_surface_band_width(eps: float, tau: float) -> float:
    return float(lib().mbo_surface_band_width(float(eps), float(tau)))


def mbo_surface_heat_modes(eps: float, tau: float, R: float):
    h, M = C.c_double(), C.c_int()
    _scheck(lib().mbo_surface_heat_modes(float(eps), float(tau), float(R), C.byref(h), C.byref(M)))
    return h.value, M.value


def mbo_surface_sphere_band(radius: float, dx: float, wb: float, p: int):
    """(xq, wq, xc) host arrays of the sphere band (count query, then fill)."""
    cnt = C.c_int64()
    _scheck(lib().mbo_surface_sphere_band(float(radius), float(dx), float(wb), int(p), None, None,
                                          None, 0, C.byref(cnt)))
    n = cnt.value
    xq, wq, xc = np.empty((n, 3)), np.empty(n), np.empty((n, 3))
    _scheck(lib().mbo_surface_sphere_band(float(radius), float(dx), float(wb), int(p), xq.ctypes.data,
                                          wq.ctypes.data, xc.ctypes.data, n, C.byref(cnt)))
    return xq, wq, xc


def mbo_surface_peanut_band(dx: float, wb: float, p: int):
    """(xq, wq, xc) host arrays of the peanut band (count query, then fill)."""
    cnt = C.c_int64()
    _scheck(lib().mbo_surface_peanut_band(float(dx), float(wb), int(p), None, None, None, 0, C.byref(cnt)))
    n = cnt.value
    xq, wq, xc = np.empty((n, 3)), np.empty(n), np.empty((n, 3))
    _scheck(lib().mbo_surface_peanut_band(float(dx), float(wb), int(p), xq.ctypes.data, wq.ctypes.data,
                                          xc.ctypes.data, n, C.byref(cnt)))
    return xq, wq, xc


def mbo_surface_create(xq, wq, xc, n: int, tau: float, eps: float, dtype: int = MBO_F32):
    xq = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    xc = np.ascontiguousarray(xc, dtype=np.float64).reshape(-1, 3)
    wq = np.ascontiguousarray(wq, dtype=np.float64).reshape(-1)
    s = C.c_void_p()
    _scheck(lib().mbo_surface_create(C.byref(s), xq.shape[0], xq.ctypes.data, wq.ctypes.data,
                                     xc.ctypes.data, int(n), float(tau), float(eps), int(dtype)))
    return s


def mbo_surface_destroy(s) -> None:
    _scheck(lib().mbo_surface_destroy(s))


def mbo_surface_get_params(s) -> dict:
    p = mbo_surface_params()
    _scheck(lib().mbo_surface_get_params(s, C.byref(p)), s)
    return p.as_dict()


def mbo_surface_diffuse(s, A, A_tilde, stream=None) -> None:
    _scheck(lib().mbo_surface_diffuse(s, _ptr(A), _ptr(A_tilde), _stream(stream)), s)


def mbo_surface_step(s, A, want_stats: bool = False, stream=None):
    st = mbo_stats()
    _scheck(lib().mbo_surface_step(s, _ptr(A), C.byref(st) if want_stats else None, _stream(stream)), s)
    return st.as_dict() if want_stats else None


def mbo_surface_step_volume(s, A, volume: float = -1.0, want_stats: bool = False, stream=None):
    st = mbo_stats()
    _scheck(lib().mbo_surface_step_volume(s, _ptr(A), float(volume), C.byref(st) if want_stats else None,
                                          _stream(stream)), s)
    return st.as_dict() if want_stats else None


def mbo_surface_profile_enable(s, enable: bool = True) -> None:
    _scheck(lib().mbo_surface_profile_enable(s, 1 if enable else 0), s)


def mbo_surface_profile_read(s) -> dict:
    """{pass: (milliseconds, timed calls)} for the passes of SURFACE_PASSES."""
    n = len(SURFACE_PASSES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _scheck(lib().mbo_surface_profile_read(s, ms, cnt, n), s)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(SURFACE_PASSES)}


def mbo_surface_workspace_bytes(s) -> int:
    return int(lib().mbo_surface_workspace_bytes(s))


class Surface:
    """Owning wrapper of a surface plan.  Fields: tensors of shape (n*n, nq)."""

    def __init__(self, xq, wq, xc, n: int, tau: float, eps: float, dtype: str = "f32"):
        self.n, self.tau, self.eps = int(n), float(tau), float(eps)
        self.nq = int(np.asarray(wq).size)
        self.dtype = {"f32": MBO_F32, "f64": MBO_F64}[dtype]
        self.h = mbo_surface_create(xq, wq, xc, n, tau, eps, self.dtype)

    def close(self) -> None:
        if getattr(self, "h", None) is not None:
            mbo_surface_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> dict:
        return mbo_surface_get_params(self.h)

    def diffuse(self, A, out, stream=None):
        mbo_surface_diffuse(self.h, A, out, stream)
        return out

    def step(self, A, want_stats=False, stream=None):
        return mbo_surface_step(self.h, A, want_stats, stream)

    def step_volume(self, A, volume: float = -1.0, want_stats=False, stream=None):
        return mbo_surface_step_volume(self.h, A, volume, want_stats, stream)
