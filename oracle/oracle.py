"""ctypes binding of the FP64 CPU oracle (``oracle/mbo_oracle.c``).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg load it; the CUDA library never does.  Every function here
marshals numpy arrays into the C routines, which follow Algorithm 1 of
Osting & Wang (arXiv:1711.01365): the diffusion step of Sec. 5.1, the
projection of Lemma 1.1, and the Lyapunov functional of Sec. 4.

Field layout: float64 array of shape ``(n*n, *dims)``, channel ``i*n+j`` holding
matrix entry ``(i, j)`` at every grid point.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbo_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmbo_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (OpenMP when available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    dp = C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_set_threads.restype = C.c_int
    lib.orc_fft.argtypes = [dp, C.c_int64, C.c_int]
    lib.orc_dft_direct.argtypes = [dp, dp, C.c_int64, C.c_int]
    lib.orc_fftn.argtypes = [dp, C.c_int, i64p, C.c_int]
    lib.orc_heat_multiplier.argtypes = [dp, C.c_int, i64p, C.c_double]
    lib.orc_diffuse.argtypes = [dp, dp, C.c_int, i64p, C.c_int, C.c_double, dp]
    lib.orc_det.argtypes = [dp, C.c_int]
    lib.orc_det.restype = C.c_double
    lib.orc_polar.argtypes = [dp, dp, dp, C.c_int]
    lib.orc_polar.restype = C.c_int
    lib.orc_project_field.argtypes = [dp, dp, C.POINTER(C.c_int8), C.c_int64, C.c_int]
    lib.orc_energy_from.argtypes = [dp, dp, C.c_int, i64p, C.c_int, C.c_double]
    lib.orc_energy_from.restype = C.c_double
    lib.orc_energy.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double]
    lib.orc_energy.restype = C.c_double
    lib.orc_energy_spectral.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double]
    lib.orc_energy_spectral.restype = C.c_double
    lib.orc_step.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double, C.c_void_p]
    lib.orc_run.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double, C.c_int, C.c_double,
                            C.POINTER(C.c_int), C.POINTER(C.c_int), dp, dp, i64p]
    lib.orc_step_points.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double, C.c_int, i64p,
                                    C.c_int64, dp, dp]
    lib.orc_polar_class.argtypes = [dp, dp, C.c_int, C.c_int]
    lib.orc_polar_class.restype = C.c_int
    lib.orc_delta_energy.argtypes = [dp, C.c_int]
    lib.orc_delta_energy.restype = C.c_double
    lib.orc_count_positive.argtypes = [dp, C.c_int64, C.c_int]
    lib.orc_count_positive.restype = C.c_int64
    lib.orc_step_volume.argtypes = [dp, C.c_int, i64p, C.c_int, C.c_double, C.c_int64, C.c_void_p, dp]
    lib.orc_step_volume.restype = C.c_int
    lib.orc_step_points_f32.argtypes = [C.POINTER(C.c_float), C.c_int, i64p, C.c_int, C.c_double,
                                        C.c_int, i64p, C.c_int64, dp, dp]
    for f in ("orc_fft", "orc_dft_direct", "orc_fftn", "orc_heat_multiplier", "orc_diffuse",
              "orc_project_field", "orc_step", "orc_run", "orc_step_points",
              "orc_step_points_f32"):
        getattr(lib, f).restype = C.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _dims(dims) -> C.Array:
    return (C.c_int64 * len(dims))(*[int(d) for d in dims])


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class OracleStats(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_delta", C.c_double), ("det_flips", C.c_int64),
                ("max_imag", C.c_double)]


def set_threads(t: int) -> int:
    """Set the OpenMP thread count (t <= 0 keeps it); returns the count in use."""
    return _load().orc_set_threads(int(t))


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 1-D DFT, exp(sign*2*pi*i*jk/N), mixed radix 2/3."""
    z = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(_load().orc_fft(_dp(z.view(np.float64)), z.size, sign), "fft")
    return z


def dft_direct(x: np.ndarray, sign: int = -1) -> np.ndarray:
    z = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(z)
    _check(_load().orc_dft_direct(_dp(z.view(np.float64)), _dp(out.view(np.float64)), z.size, sign),
           "dft_direct")
    return out


def fftn(x: np.ndarray, sign: int = -1) -> np.ndarray:
    z = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(_load().orc_fftn(_dp(z.view(np.float64)), z.ndim, _dims(z.shape), sign), "fftn")
    return z


def heat_multiplier(dims, tau: float) -> np.ndarray:
    g = np.empty(tuple(dims), dtype=np.float64)
    _check(_load().orc_heat_multiplier(_dp(g), len(dims), _dims(dims), float(tau)), "multiplier")
    return g


def diffuse(A: np.ndarray, tau: float, return_max_imag: bool = False):
    """e^{tau Delta} applied channel by channel; A has shape (C, *dims)."""
    A = _f64(A)
    out = np.empty_like(A)
    mi = C.c_double(0.0)
    _check(_load().orc_diffuse(_dp(A), _dp(out), A.ndim - 1, _dims(A.shape[1:]), A.shape[0],
                               float(tau), C.byref(mi)), "diffuse")
    return (out, mi.value) if return_max_imag else out


def det(M: np.ndarray) -> float:
    M = _f64(M)
    return _load().orc_det(_dp(M), M.shape[0])


def polar(M: np.ndarray, return_sigma: bool = False):
    """Closest orthogonal matrix of one n x n matrix (Lemma 1.1)."""
    M = _f64(M)
    n = M.shape[0]
    B = np.empty_like(M)
    s = np.empty(n, dtype=np.float64)
    rc = _load().orc_polar(_dp(M), _dp(B), _dp(s), n)
    if rc < 0:
        raise RuntimeError("oracle polar failed")
    return (B, s) if return_sigma else B


def project(At: np.ndarray, n: int, return_sign: bool = False):
    """Project every grid point of a planar field (shape (n*n, *dims))."""
    At = _f64(At)
    P = int(np.prod(At.shape[1:])) if At.ndim > 1 else 1
    B = np.empty_like(At)
    sg = np.empty(At.shape[1:], dtype=np.int8)
    _check(_load().orc_project_field(_dp(At), _dp(B), sg.ctypes.data_as(C.POINTER(C.c_int8)), P, n),
           "project")
    return (B, sg) if return_sign else B


def energy_from(A: np.ndarray, At: np.ndarray, n: int, tau: float) -> float:
    A, At = _f64(A), _f64(At)
    return _load().orc_energy_from(_dp(A), _dp(At), A.ndim - 1, _dims(A.shape[1:]), n, float(tau))


def energy(A: np.ndarray, n: int, tau: float) -> float:
    """E^tau(A), physical form (Sec. 4 functional with weight prod h_j)."""
    A = _f64(A)
    return _load().orc_energy(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau))


def energy_spectral(A: np.ndarray, n: int, tau: float) -> float:
    """E^tau(A), Parseval form with 1 - g computed as -expm1."""
    A = _f64(A)
    return _load().orc_energy_spectral(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau))


def step(A: np.ndarray, n: int, tau: float):
    """One iteration of Algorithm 1; returns (A_next, stats dict)."""
    A = _f64(A).copy()
    st = OracleStats()
    _check(_load().orc_step(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau), C.byref(st)),
           "step")
    return A, {"energy": st.energy, "max_delta": st.max_delta, "det_flips": st.det_flips,
               "max_imag": st.max_imag}


def step_points(A: np.ndarray, n: int, tau: float, pts, project_input: bool = False):
    """One step evaluated only at the grid points pts (array (npts, ndim) of
    indices), from the convolution definition of the diffusion; with
    project_input the raw field A is projected first.  Returns (A~, B) at the
    points, each of shape (npts, n*n)."""
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    npts = pts.shape[0]
    At = np.empty((npts, n * n))
    B = np.empty((npts, n * n))
    pp = pts.ctypes.data_as(C.POINTER(C.c_int64))
    if isinstance(A, np.ndarray) and A.dtype == np.float32 and A.flags.c_contiguous:
        rc = _load().orc_step_points_f32(A.ctypes.data_as(C.POINTER(C.c_float)), A.ndim - 1,
                                         _dims(A.shape[1:]), n, float(tau),
                                         1 if project_input else 0, pp, npts, _dp(At), _dp(B))
    else:
        A = _f64(A)
        rc = _load().orc_step_points(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau),
                                     1 if project_input else 0, pp, npts, _dp(At), _dp(B))
    _check(rc, "step_points")
    return At, B


def polar_class(M: np.ndarray, cls: int) -> np.ndarray:
    """Closest matrix of SO(n) (cls = +1) or SO^-(n) (cls = -1), Lemma 7.1."""
    M = _f64(M)
    B = np.empty_like(M)
    _load().orc_polar_class(_dp(M), _dp(B), M.shape[0], int(cls))
    return B


def delta_energy(M: np.ndarray) -> float:
    """<T+(M) - T-(M), M>_F (Sec. 7)."""
    M = _f64(M)
    return _load().orc_delta_energy(_dp(M), M.shape[0])


def count_positive(A: np.ndarray, n: int) -> int:
    A = _f64(A)
    return int(_load().orc_count_positive(_dp(A), int(np.prod(A.shape[1:])), n))


def step_volume(A: np.ndarray, n: int, tau: float, n_plus: int = -1):
    """One volume-preserving step (Sec. 7); returns (A_next, stats, dE)."""
    A = _f64(A).copy()
    st = OracleStats()
    dE = np.empty(A.shape[1:])
    _check(_load().orc_step_volume(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau),
                                   int(n_plus), C.byref(st), _dp(dE)), "step_volume")
    return A, {"energy": st.energy, "max_delta": st.max_delta, "det_flips": st.det_flips}, dE


def run(A: np.ndarray, n: int, tau: float, max_steps: int, tol: float):
    """Iterate to stationarity (or max_steps).  Returns (A_final, info dict)."""
    A = _f64(A).copy()
    steps = C.c_int(0)
    stat = C.c_int(0)
    en = np.zeros(max_steps + 1, dtype=np.float64)
    md = np.zeros(max(max_steps, 1), dtype=np.float64)
    fl = np.zeros(max(max_steps, 1), dtype=np.int64)
    _check(_load().orc_run(_dp(A), A.ndim - 1, _dims(A.shape[1:]), n, float(tau), int(max_steps),
                           float(tol), C.byref(steps), C.byref(stat), _dp(en), _dp(md),
                           fl.ctypes.data_as(C.POINTER(C.c_int64))), "run")
    s = steps.value
    return A, {"steps": s, "stationary": bool(stat.value), "energies": en[: s + 1],
               "max_deltas": md[:s], "det_flips": fl[:s]}


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
