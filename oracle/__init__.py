"""FP64 CPU oracle for the 3-D heat diffusion step (arXiv 2211.15634, Fig. 1).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports, links or executes anything here, and nothing here imports the CUDA
library.  The arithmetic lives in ``diffusion3d_oracle.c`` (plain C, FP64,
compiled without FMA contraction); this module compiles it with gcc and
wraps it with ctypes over C-contiguous float64 numpy arrays of shape
``(nz, ny, nx)``.

Entry points and the passages they follow:

* :func:`maximum`, :func:`stable_dt` - Fig. 1, the ``dt`` line.
* :func:`step` - Fig. 1, ``step!`` (interior nodes only).
* :func:`run` - Fig. 1 time loop: ``T2 = copy(T)``, then step and swap.
* :func:`adjoint_step` - transpose of one ``step!`` (derived, no paper line).
* :func:`gradient` - L = 1/2||T(nt)-T_obs||^2 and its gradient in T0 and Ci.
* :func:`stable_dt2d`, :func:`step2d`, :func:`run2d` - the 2-D form of Fig. 1's ``step!`` (the z term
  dropped; arrays of shape ``(ny, nx)``), its ``dt`` and its time loop.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diffusion3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no FMA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.or_set_threads.argtypes = [i32]
            lib.or_get_threads.restype = i32
            lib.or_max_threads.restype = i32
            lib.or_maximum.argtypes = [p, i64]
            lib.or_maximum.restype = d
            lib.or_stable_dt.argtypes = [d, d, d, d, d]
            lib.or_stable_dt.restype = d
            lib.or_stable_dt2d.argtypes = [d, d, d, d]
            lib.or_stable_dt2d.restype = d
            lib.or_step.argtypes = [p, p, p, d, d, d, d, d, i64, i64, i64]
            lib.or_run.argtypes = [p, p, p, d, d, d, d, d, i64, i64, i64, i32]
            lib.or_step_explicit.argtypes = [p, p, p, d, d, d, d, d, i64, i64, i64]
            lib.or_run_explicit.argtypes = [p, p, p, d, d, d, d, d, i64, i64, i64, i32]
            lib.or_run.restype = i32
            lib.or_adjoint_step.argtypes = [p, p, p, p, p, d, d, d, d, d, i64, i64, i64]
            lib.or_gradient.argtypes = [p, p, p, p, p, d, d, d, d, d, i64, i64, i64, i32]
            lib.or_gradient.restype = d
            lib.or_step2d.argtypes = [p, p, p, d, d, d, d, i64, i64]
            lib.or_run2d.argtypes = [p, p, p, d, d, d, d, i64, i64, i32]
            lib.or_run2d.restype = i32
            _lib = lib
    return _lib


def _f64(a: np.ndarray, name: str) -> np.ndarray:
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.ndim != 3:
        raise ValueError(f"{name}: need a C-contiguous float64 array of shape (nz, ny, nx)")
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def set_threads(n: int) -> None:
    """Host threads for the step loops (OpenMP over z; 1 = serial)."""
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return _load().or_get_threads()


def max_threads() -> int:
    return _load().or_max_threads()


def maximum(A: np.ndarray) -> float:
    """``maximum(Ci)`` (Fig. 1)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    return _load().or_maximum(_ptr(A), A.size)


def stable_dt(dx: float, dy: float, dz: float, lam: float, maxCi: float) -> float:
    """``dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1`` (Fig. 1)."""
    return _load().or_stable_dt(dx, dy, dz, lam, maxCi)


def step(T2: np.ndarray, T: np.ndarray, Ci: np.ndarray, lam: float, dt: float,
         _dx: float, _dy: float, _dz: float, *, explicit: bool = False) -> None:
    """``step!(T2, T, Ci, lam, dt, _dx, _dy, _dz)`` of Fig. 1, in place on T2's interior
    (``explicit``: in the explicit notation, see :func:`run`)."""
    for a, nm in ((T2, "T2"), (T, "T"), (Ci, "Ci")):
        _f64(a, nm)
    nz, ny, nx = T.shape
    fn = _load().or_step_explicit if explicit else _load().or_step
    fn(_ptr(T2), _ptr(T), _ptr(Ci), lam, dt, _dx, _dy, _dz, nx, ny, nz)


def run(T0: np.ndarray, Ci: np.ndarray, lam: float, dt: float, _dx: float, _dy: float,
        _dz: float, nt: int, *, explicit: bool = False) -> np.ndarray:
    """Fig. 1 time loop from T0 for nt steps; returns the final state (a new array).
    ``explicit``: the step in the explicit notation of the paper's Results (second
    differences A[i+1] - 2*A[i] + A[i-1]) instead of Fig. 1's @d2_xi form."""
    T = np.array(_f64(T0, "T0"), copy=True)
    T2 = np.empty_like(T)
    _f64(Ci, "Ci")
    nz, ny, nx = T.shape
    fn = _load().or_run_explicit if explicit else _load().or_run
    odd = fn(_ptr(T), _ptr(T2), _ptr(Ci), lam, dt, _dx, _dy, _dz, nx, ny, nz, int(nt))
    return T2 if odd else T


def adjoint_step(ybar: np.ndarray, T: np.ndarray, Ci: np.ndarray, Cibar: np.ndarray, lam: float,
                 dt: float, _dx: float, _dy: float, _dz: float) -> np.ndarray:
    """Transpose of one step: returns ``Tbar``; adds this step's term into ``Cibar`` in place."""
    for a, nm in ((ybar, "ybar"), (T, "T"), (Ci, "Ci"), (Cibar, "Cibar")):
        _f64(a, nm)
    nz, ny, nx = T.shape
    Tbar = np.empty_like(T)
    _load().or_adjoint_step(_ptr(Tbar), _ptr(Cibar), _ptr(ybar), _ptr(T), _ptr(Ci), lam, dt,
                            _dx, _dy, _dz, nx, ny, nz)
    return Tbar


def gradient(T0: np.ndarray, Ci: np.ndarray, Tobs: np.ndarray, lam: float, dt: float,
             _dx: float, _dy: float, _dz: float, nt: int):
    """``(L, dL/dT0, dL/dCi)`` for ``L = 1/2 ||T(nt) - Tobs||^2`` with dt held fixed."""
    for a, nm in ((T0, "T0"), (Ci, "Ci"), (Tobs, "Tobs")):
        _f64(a, nm)
    nz, ny, nx = T0.shape
    dT0 = np.empty_like(T0)
    dCi = np.empty_like(T0)
    L = _load().or_gradient(_ptr(dT0), _ptr(dCi), _ptr(T0), _ptr(Ci), _ptr(Tobs), lam, dt,
                            _dx, _dy, _dz, nx, ny, nz, int(nt))
    if L < 0:
        raise MemoryError("oracle gradient: out of host memory for the stored states")
    return L, dT0, dCi


def loss(T: np.ndarray, Tobs: np.ndarray) -> float:
    """``1/2 ||T - Tobs||^2`` in FP64 (numpy dot of the residual)."""
    r = (T - Tobs).ravel()
    return 0.5 * float(np.dot(r, r))


def stable_dt2d(dx: float, dy: float, lam: float, maxCi: float) -> float:
    """2-D form of Fig. 1's ``dt`` line: ``min(dx^2,dy^2)/lam/maximum(Ci)/4.1``."""
    return _load().or_stable_dt2d(dx, dy, lam, maxCi)


def _f64_2d(a: np.ndarray, name: str) -> np.ndarray:
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.ndim != 2:
        raise ValueError(f"{name}: need a C-contiguous float64 array of shape (ny, nx)")
    return a


def step2d(T2: np.ndarray, T: np.ndarray, Ci: np.ndarray, lam: float, dt: float, _dx: float,
           _dy: float) -> None:
    """2-D form of Fig. 1's ``step!`` (z term dropped), in place on T2's interior."""
    for a, nm in ((T2, "T2"), (T, "T"), (Ci, "Ci")):
        _f64_2d(a, nm)
    ny, nx = T.shape
    _load().or_step2d(_ptr(T2), _ptr(T), _ptr(Ci), lam, dt, _dx, _dy, nx, ny)


def run2d(T0: np.ndarray, Ci: np.ndarray, lam: float, dt: float, _dx: float, _dy: float,
          nt: int) -> np.ndarray:
    """2-D time loop from T0 for nt steps; returns the final state (a new array)."""
    T = np.array(_f64_2d(T0, "T0"), copy=True)
    T2 = np.empty_like(T)
    _f64_2d(Ci, "Ci")
    ny, nx = T.shape
    odd = _load().or_run2d(_ptr(T), _ptr(T2), _ptr(Ci), lam, dt, _dx, _dy, nx, ny, int(nt))
    return T2 if odd else T
