"""ctypes binding of ``libpsdiff.so`` (the C ABI in ``include/ps_diffusion3d.h``).

Only argument marshalling lives here: every operation runs in the library's
CUDA kernels.  Loading fails loudly if the library cannot be built or
loaded - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PS_F32 = 0
PS_F64 = 1
PS_OK = 0
PS_ERR_ARG = -1
PS_ERR_ALIAS = -2
PS_ERR_ALIGN = -3
PS_ERR_CUDA = -4
PS_ERR_UNSUPPORTED = -5
PS_RUN_GRAPH = 1
PS_RUN_COMPENSATED = 2
PS_RUN_NATIVE_F64 = 4
PS_RUN_CI_SCALED = 8
PS_RUN_TEMPORAL2 = 16
PS_BATCH_COLUMN = 1
PS_BATCH_ZMARCH = 2
PS_BATCH_CI_SCALED = 4
PS_BATCH_TEMPORAL2 = 8
PS_OVERRIDE = {"kchunk": 0, "kchunk2": 1, "adj_kchunk": 2, "chunk2d": 3, "adj_plain": 4, "f64_px2": 5,
               "step_plain": 6}

STATUS_NAMES = {0: "PS_OK", -1: "PS_ERR_ARG", -2: "PS_ERR_ALIAS", -3: "PS_ERR_ALIGN",
                -4: "PS_ERR_CUDA", -5: "PS_ERR_UNSUPPORTED"}


class PsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PsProblem(ctypes.Structure):
    _fields_ = [("T", ctypes.c_void_p), ("T2", ctypes.c_void_p), ("Ci", ctypes.c_void_p),
                ("lam", ctypes.c_double), ("dt", ctypes.c_double), ("_dx", ctypes.c_double),
                ("_dy", ctypes.c_double), ("_dz", ctypes.c_double), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("tile_x", ctypes.c_int32),
                ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32), ("pitch", ctypes.c_int32)]


# name -> (restype, argtypes)
_P, _D, _I64, _I, _U, _SZ = (ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                             ctypes.c_uint, ctypes.c_size_t)
SIGNATURES = {
    "ps_version": (_I, []),
    "ps_last_error": (ctypes.c_char_p, []),
    "ps_workspace_bytes": (_SZ, []),
    "ps_device_error": (_I, [ctypes.POINTER(_U), _I]),
    "ps_selftest_bounded_wait": (_I, [_U, _U, _P]),
    "ps_diffusion3d_step_kernel": (ctypes.c_char_p, [_P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I,
                                                     _U]),
    "ps_diffusion3d_step_ex": (_I, [_P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _U, _P]),
    "ps_diffusion3d_scale_ci": (_I, [_P, _P, _D, _D, _D, _I64, _P]),
    "ps_diffusion3d_step": (_I, [_P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _P]),
    "ps_diffusion3d_step_comp_f32": (_I, [_P, _P, _P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _P]),
    "ps_to_deviation_pair": (_I, [_P, _P, _P, _D, _I64, _P]),
    "ps_from_deviation_pair": (_I, [_P, _P, _P, _D, _I64, _P]),
    "ps_diffusion3d_copy_boundary": (_I, [_P, _P, _I64, _I64, _I64, _I, _P]),
    "ps_diffusion3d_copy_boundary_many": (_I, [_P, _I64, _I64, _P, _I64, _I64, _I64, _I, _P]),
    "ps_diffusion3d_run": (_I, [_P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _I, _P,
                                ctypes.POINTER(_I)]),
    "ps_diffusion3d_run_ex": (_I, [_P, _P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _I, _U,
                                   _P, ctypes.POINTER(_I)]),
    "ps_diffusion3d_run_states": (_I, [_P, _P, _I64, _I, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I,
                                       _I, _U, _P, ctypes.POINTER(_I)]),
    "ps_clear_graph_cache": (_I, []),
    "ps_graph_cache_size": (_SZ, []),
    "ps_set_launch_override": (_I, [_I, _I]),
    "ps_get_launch_override": (_I, [_I, ctypes.POINTER(_I)]),
    "ps_diffusion2d_stable_dt": (_I, [ctypes.POINTER(_D), _P, _I64, _I64, _D, _D, _D, _I, _P, _P]),
    "ps_diffusion3d_adjoint": (_I, [_P, _P, _P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _P]),
    "ps_diffusion3d_adjoint_ex": (_I, [_P, _P, _P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I,
                                       _U, _P]),
    "ps_maximum_async": (_I, [_P, _P, _I64, _I, _P, _P]),
    "ps_maximum": (_I, [ctypes.POINTER(_D), _P, _I64, _I, _P, _P]),
    "ps_diffusion3d_stable_dt": (_I, [ctypes.POINTER(_D), _P, _I64, _I64, _I64, _D, _D, _D, _D, _I,
                                      _P, _P]),
    "ps_dot": (_I, [_P, _P, _P, _I64, _I, _P, _P]),
    "ps_dot_static": (_I, [_P, _P, _P, _I64, _I, _P]),
    "ps_half_sq_dist": (_I, [_P, _P, _P, _P, _I64, _I, _P, _P]),
    "ps_to_deviation": (_I, [_P, _P, _D, _I64, _P]),
    "ps_from_deviation": (_I, [_P, _P, _D, _I64, _P]),
    "ps_batch_table_bytes": (_SZ, [ctypes.POINTER(PsProblem), _I, _I, _I, _I, _I]),
    "ps_batch_table_fill": (_I, [_P, _SZ, ctypes.POINTER(PsProblem), _I, _I, _I, _I, _I,
                                 ctypes.POINTER(_I64)]),
    "ps_diffusion3d_batch_step": (_I, [_P, _I, _I, _P]),
    "ps_diffusion3d_batch_run": (_I, [_P, _I, _I, _U, _P]),
    "ps_batch_table_bytes_ex": (_SZ, [ctypes.POINTER(PsProblem), _I, _I, _I, _I, _I, _U]),
    "ps_batch_table_fill_ex": (_I, [_P, _SZ, ctypes.POINTER(PsProblem), _I, _I, _I, _I, _I, _U,
                                    ctypes.POINTER(_I64)]),
    "ps_batch_table_kernel": (_I, [_P]),
    "ps_diffusion3d_batch_step_ex": (_I, [_P, _P, _I, _P]),
    "ps_diffusion2d_step": (_I, [_P, _P, _P, _D, _D, _D, _D, _I64, _I64, _I, _U, _P]),
    "ps_diffusion2d_run": (_I, [_P, _P, _P, _D, _D, _D, _D, _I64, _I64, _I, _I, _U, _P, ctypes.POINTER(_I)]),
    "ps_diffusion3d_adjoint2_ex": (_I, [_P, _P, _P, _P, _P, _P, _D, _D, _D, _D, _D, _I64, _I64, _I64, _I, _U,
                                        _P]),
    "ps_diffusion3d_batch_step2_ex": (_I, [_P, _P, _I, _P]),
    "ps_diffusion3d_batch_run_ex": (_I, [_P, _P, _I, _U, _P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load (building first if needed) and return the ctypes library handle."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not found at {path}; run build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int) -> None:
    """Raise PsError for a non-OK status, with the library's message."""
    if status != PS_OK:
        msg = load().ps_last_error()
        raise PsError(status, msg.decode() if msg else "")
