"""C-ABI checks that need no GPU: the library loads, exports every symbol
declared in include/*.h, and rejects bad arguments on the host before any
launch (fake device addresses are never dereferenced)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2211_15634_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ps_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ps_diffusion3d_step", "ps_diffusion3d_run", "ps_diffusion3d_adjoint",
                 "ps_diffusion3d_batch_step", "ps_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert set(_lib.SIGNATURES) >= set(declared_functions())


def test_version_and_workspace(lib):
    assert lib.ps_version() >= 100
    assert lib.ps_workspace_bytes() >= 8 * 1024 + 64


A = 0x10000       # fake, 16-byte aligned device addresses (never dereferenced)
B = 0x90000000
C = 0x190000000


def step(lib, T2=B, T=A, Ci=C, n=(8, 8, 8), dtype=_lib.PS_F64, dt=1e-3):
    return lib.ps_diffusion3d_step(T2, T, Ci, 1.0, dt, 7.0, 7.0, 7.0, *n, dtype, None)


@pytest.mark.parametrize("kw,status", [
    (dict(T2=None), _lib.PS_ERR_ARG),
    (dict(T=None), _lib.PS_ERR_ARG),
    (dict(Ci=None), _lib.PS_ERR_ARG),
    (dict(n=(2, 8, 8)), _lib.PS_ERR_ARG),
    (dict(n=(8, 8, 0)), _lib.PS_ERR_ARG),
    (dict(dtype=7), _lib.PS_ERR_ARG),
    (dict(dt=float("nan")), _lib.PS_ERR_ARG),
    (dict(T2=A), _lib.PS_ERR_ALIAS),
    (dict(T2=A + 16), _lib.PS_ERR_ALIAS),
    (dict(T2=C), _lib.PS_ERR_ALIAS),
    (dict(T=A + 8), _lib.PS_ERR_ALIGN),
])
def test_step_rejects_bad_arguments(lib, kw, status):
    assert step(lib, **kw) == status
    assert len(lib.ps_last_error()) > 0


def test_last_error_names_the_argument(lib):
    assert step(lib, Ci=None) == _lib.PS_ERR_ARG
    assert b"Ci" in lib.ps_last_error()
    assert step(lib, n=(8, 1, 8)) == _lib.PS_ERR_ARG
    assert b">= 3" in lib.ps_last_error()


def test_run_and_adjoint_reject_bad_arguments(lib):
    odd = ctypes.c_int(-1)
    assert lib.ps_diffusion3d_run(A, B, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, -1, _lib.PS_F64, None,
                                  ctypes.byref(odd)) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_run_ex(A, B, None, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, 3, _lib.PS_F64,
                                     _lib.PS_RUN_COMPENSATED, None, ctypes.byref(odd)) == _lib.PS_ERR_UNSUPPORTED
    assert lib.ps_diffusion3d_run_ex(A, B, None, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, 3, _lib.PS_F32,
                                     _lib.PS_RUN_COMPENSATED, None, ctypes.byref(odd)) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_run_ex(A, B, None, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, 3, _lib.PS_F64,
                                     0x100, None, ctypes.byref(odd)) == _lib.PS_ERR_ARG
    D, E = 0x290000000, 0x390000000
    # Tbar overlapping ybar, Cibar overlapping T
    assert lib.ps_diffusion3d_adjoint(A, B, A, C, D, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8,
                                      _lib.PS_F64, None) == _lib.PS_ERR_ALIAS
    assert lib.ps_diffusion3d_adjoint(E, C, A, C, D, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8,
                                      _lib.PS_F64, None) == _lib.PS_ERR_ALIAS
    assert lib.ps_diffusion3d_adjoint(E, B, A, C, None, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8,
                                      _lib.PS_F64, None) == _lib.PS_ERR_ARG


def test_reductions_reject_bad_arguments(lib):
    v = ctypes.c_double(0)
    assert lib.ps_maximum(ctypes.byref(v), A, 0, _lib.PS_F64, B, None) == _lib.PS_ERR_ARG
    assert lib.ps_maximum(ctypes.byref(v), A, 10, _lib.PS_F64, None, None) == _lib.PS_ERR_ARG
    assert lib.ps_maximum(None, A, 10, _lib.PS_F64, B, None) == _lib.PS_ERR_ARG
    assert lib.ps_dot(None, A, B, 10, _lib.PS_F64, C, None) == _lib.PS_ERR_ARG
    assert lib.ps_half_sq_dist(C, A, A, B, 10, _lib.PS_F64, C + 4096, None) == _lib.PS_ERR_ALIAS
    assert lib.ps_diffusion3d_batch_step(None, 0, _lib.PS_F64, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_step(A, 2, _lib.PS_F64, None) == _lib.PS_ERR_ARG


def make_problems(sizes, base=0x100000000, pitch=0):
    arr = (_lib.PsProblem * len(sizes))()
    addr = base
    for q, n in enumerate(sizes):
        nbytes = ((pitch or n) * n * n * 8 + 4095) // 4096 * 4096
        T, T2, Ci = addr, addr + nbytes, addr + 2 * nbytes
        addr += 3 * nbytes
        arr[q] = _lib.PsProblem(T, T2, Ci, 1.0, 1e-4, n - 1.0, n - 1.0, n - 1.0, n, n, n, 0, 0, 0, pitch)
    return arr


ITEM = [("prob", "<i4"), ("i0", "<i4"), ("j0", "<i4"), ("k0", "<i4"), ("ni", "<i2"), ("nj", "<i2"),
        ("nk", "<i2"), ("kind", "<i2")]


@pytest.mark.parametrize("own_tile", [False, True])
def test_batch_table_layout(lib, own_tile):
    """The column-march table lists every interior node exactly once, largest
    items first; a problem's own tile fields override the call's tile."""
    import numpy as np
    sizes = [5, 33, 17, 40]
    arr = make_problems(sizes)
    tx, ty, tz = 8, 4, 6
    if own_tile:
        arr[3].tile_x, arr[3].tile_y, arr[3].tile_z = 16, 3, 7
    nbytes = lib.ps_batch_table_bytes(arr, len(sizes), _lib.PS_F64, tx, ty, tz)
    assert nbytes > 0
    buf = (ctypes.c_char * nbytes)()
    nitems = ctypes.c_int64(0)
    assert lib.ps_batch_table_fill(buf, nbytes, arr, len(sizes), _lib.PS_F64, tx, ty, tz,
                                   ctypes.byref(nitems)) == _lib.PS_OK
    raw = bytes(buf)
    nprob, nit = np.frombuffer(raw[:16], dtype=np.int64)
    dtype, ttx, tty, ttz = np.frombuffer(raw[16:32], dtype=np.int32)
    poff, ioff = np.frombuffer(raw[32:48], dtype=np.int64)
    assert (nprob, nit, dtype, ttx, tty, ttz) == (4, nitems.value, _lib.PS_F64, tx, ty, tz)
    items = np.frombuffer(raw[ioff:ioff + 24 * nit], dtype=np.dtype(ITEM))
    covered = {q: np.zeros((n, n, n), dtype=np.int32) for q, n in enumerate(sizes)}
    works = []
    for it in items:
        q, i0, j0, k0 = int(it["prob"]), int(it["i0"]), int(it["j0"]), int(it["k0"])
        n = sizes[q]
        px, py, pz = (16, 3, 7) if (own_tile and q == 3) else (tx, ty, tz)
        i1, j1, k1 = min(i0 + px, n - 1), min(j0 + py, n - 1), min(k0 + pz, n - 1)
        assert (it["ni"], it["nj"], it["nk"]) == (i1 - i0, j1 - j0, k1 - k0)
        covered[q][k0:k1, j0:j1, i0:i1] += 1
        works.append((i1 - i0) * (j1 - j0) * (k1 - k0))
    for q, n in enumerate(sizes):
        inner = covered[q][1:-1, 1:-1, 1:-1]
        assert inner.min() == 1 and inner.max() == 1
        assert covered[q].sum() == (n - 2) ** 3
    assert works == sorted(works, reverse=True)
    # problem records carry the pointers and step coefficients
    rec = np.frombuffer(raw[poff:poff + 80], dtype=np.uint64)
    assert int(rec[0]) == arr[0].T and int(rec[1]) == arr[0].T2 and int(rec[2]) == arr[0].Ci


def test_batch_table_rejects_bad_problem(lib):
    arr = make_problems([8, 9])
    arr[1].T2 = arr[1].T  # aliasing inside one problem
    nbytes = lib.ps_batch_table_bytes(arr, 2, _lib.PS_F64, 0, 0, 0)
    buf = (ctypes.c_char * nbytes)()
    assert lib.ps_batch_table_fill(buf, nbytes, arr, 2, _lib.PS_F64, 0, 0, 0, None) == _lib.PS_ERR_ALIAS
    assert b"problem 1" in lib.ps_last_error()
    arr = make_problems([8])
    assert lib.ps_batch_table_fill(buf, 16, arr, 1, _lib.PS_F64, 0, 0, 0, None) == _lib.PS_ERR_ARG


def test_prescaled_step_rejects_fp32_anisotropic_and_unknown_flags(lib):
    S = _lib.PS_RUN_CI_SCALED

    def step_ex(inv=(7.0, 7.0, 7.0), dtype=_lib.PS_F64, flags=S):
        return lib.ps_diffusion3d_step_ex(B, A, C, 1.0, 1e-3, *inv, 8, 8, 8, dtype, flags, None)

    assert step_ex(dtype=_lib.PS_F32) == _lib.PS_ERR_UNSUPPORTED
    assert step_ex(inv=(7.0, 7.0, 8.0)) == _lib.PS_ERR_UNSUPPORTED
    assert b"equal spacings" in lib.ps_last_error()
    assert step_ex(flags=0x40) == _lib.PS_ERR_ARG
    odd = ctypes.c_int(-1)
    assert lib.ps_diffusion3d_run_ex(A, B, None, C, 1.0, 1e-3, 7.0, 6.0, 7.0, 8, 8, 8, 3,
                                     _lib.PS_F64, S, None, ctypes.byref(odd)) == _lib.PS_ERR_UNSUPPORTED
    assert lib.ps_diffusion3d_scale_ci(B, A, 1.0, 1e-3, 7.0, 0, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_scale_ci(None, A, 1.0, 1e-3, 7.0, 10, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_scale_ci(A + 16, A, 1.0, 1e-3, 7.0, 10, None) == _lib.PS_ERR_ALIAS
    assert lib.ps_diffusion3d_scale_ci(B, A, 1.0, float("inf"), 7.0, 10, None) == _lib.PS_ERR_ARG


def test_kernel_names_for_the_fp64_step(lib):
    name = lambda nx, flags: lib.ps_diffusion3d_step_kernel(B, A, C, 1.0, 1e-3, 7.0, 7.0, 7.0, nx, 8,
                                                            8, _lib.PS_F64, flags).decode()
    # the TMA kernel needs the driver's tensor-map encoder (absent without a GPU driver)
    tma = name(64, 0) == "k_zmarch<F64_EMU_ISO>"
    assert name(64, 0) == ("k_zmarch<F64_EMU_ISO>" if tma else "k_step_basic_emu")
    assert name(64, _lib.PS_RUN_CI_SCALED) == ("k_zmarch<F64_SCALED4>" if tma else "k_step_basic_emu")
    assert name(66, _lib.PS_RUN_CI_SCALED) == ("k_zmarch<F64_SCALED>" if tma else "k_step_basic_emu")
    assert name(63, _lib.PS_RUN_CI_SCALED) == "k_step_basic_emu"


def test_scaled_adjoint_rejects_fp32_anisotropic_and_unknown_flags(lib):
    D, E = 0x290000000, 0x390000000
    S = _lib.PS_RUN_CI_SCALED

    def adj(inv=(7.0, 7.0, 7.0), dtype=_lib.PS_F64, flags=S):
        return lib.ps_diffusion3d_adjoint_ex(E, B, A, C, D, 1.0, 1e-3, *inv, 8, 8, 8, dtype, flags, None)

    assert adj(dtype=_lib.PS_F32) == _lib.PS_ERR_UNSUPPORTED
    assert adj(inv=(7.0, 6.0, 7.0)) == _lib.PS_ERR_UNSUPPORTED
    assert adj(flags=_lib.PS_RUN_GRAPH) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_adjoint_ex(A, B, A, C, D, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8,
                                         _lib.PS_F64, S, None) == _lib.PS_ERR_ALIAS


def test_temporal2_rejects_unsupported_modes(lib):
    odd = ctypes.c_int(-1)
    T2F = _lib.PS_RUN_TEMPORAL2

    def run(dtype, flags, comp=None):
        return lib.ps_diffusion3d_run_ex(A, B, comp, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, 4, dtype,
                                         flags, None, ctypes.byref(odd))

    assert run(_lib.PS_F64, T2F) == _lib.PS_ERR_UNSUPPORTED
    assert run(_lib.PS_F64, T2F | _lib.PS_RUN_NATIVE_F64) == _lib.PS_ERR_UNSUPPORTED
    assert run(_lib.PS_F32, T2F | _lib.PS_RUN_COMPENSATED, comp=0x490000000) == _lib.PS_ERR_UNSUPPORTED
    assert b"TEMPORAL2" in lib.ps_last_error()
    assert run(_lib.PS_F64, 0x40) == _lib.PS_ERR_ARG


def test_run_states_temporal2_is_fp32_only(lib):
    """The state-keeping loop takes PS_RUN_TEMPORAL2 for FP32 only (any interval); the
    refusal comes before anything is launched."""
    slot = ctypes.c_int(-9)
    for every in (1, 3):
        st = lib.ps_diffusion3d_run_states(A, B, 512, every, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 8, 8, 8, 6,
                                           _lib.PS_F64, _lib.PS_RUN_TEMPORAL2, None, ctypes.byref(slot))
        assert st == _lib.PS_ERR_UNSUPPORTED
        assert b"TEMPORAL2" in lib.ps_last_error()
    assert slot.value == -9  # nothing written


def test_copy_boundary_many_rejects_bad_stride_and_overlap(lib):
    many = lib.ps_diffusion3d_copy_boundary_many
    assert many(B, 3, 511, A, 8, 8, 8, _lib.PS_F64, None) == _lib.PS_ERR_ARG   # < nx*ny*nz
    assert many(B, 3, 514, A, 8, 8, 8, _lib.PS_F32, None) == _lib.PS_ERR_ARG   # not 16-byte
    assert many(B, 0, 512, A, 8, 8, 8, _lib.PS_F64, None) == _lib.PS_ERR_ARG
    assert many(A, 3, 512, A + 4096, 8, 8, 8, _lib.PS_F64, None) == _lib.PS_ERR_ALIAS


def test_selftest_rejects_out_of_range_arguments(lib):
    assert lib.ps_selftest_bounded_wait(0, 1000, None) == _lib.PS_ERR_ARG
    assert lib.ps_selftest_bounded_wait((1 << 24) + 1, 1000, None) == _lib.PS_ERR_ARG
    assert lib.ps_selftest_bounded_wait(16, 0, None) == _lib.PS_ERR_ARG
    assert lib.ps_selftest_bounded_wait(16, 2000000, None) == _lib.PS_ERR_ARG


def have_driver(lib):
    """True when the library can encode tensor maps (a GPU driver is present)."""
    return lib.ps_diffusion3d_step_kernel(B, A, C, 1.0, 1e-3, 7.0, 7.0, 7.0, 64, 8, 8, _lib.PS_F64,
                                          0).decode().startswith("k_zmarch")


def test_batch_pitch_and_flags(lib):
    """Row pitch in the problem records; pitch below nx, conflicting or unknown
    flags, and PS_BATCH_CI_SCALED outside FP64 z-march tables are refused; without
    a GPU driver (no tensor-map encoder) the automatic choice is the column march
    and an explicit z-march request is refused."""
    import numpy as np
    arr = make_problems([9, 12], pitch=16)
    nbytes = lib.ps_batch_table_bytes_ex(arr, 2, _lib.PS_F64, 0, 0, 0, 0)
    assert nbytes > 0
    buf = (ctypes.c_char * (nbytes + 64))()
    off = (-ctypes.addressof(buf)) % 64
    host = (ctypes.c_char * nbytes).from_buffer(buf, off)
    assert lib.ps_batch_table_fill_ex(host, nbytes, arr, 2, _lib.PS_F64, 0, 0, 0, 0, None) == _lib.PS_OK
    raw = bytes(host)
    poff = int(np.frombuffer(raw[32:40], dtype=np.int64)[0])
    if lib.ps_batch_table_kernel(host) == 0:  # the column record: 3 pointers, 4 doubles, nx ny nz, pitch
        rec = np.frombuffer(raw[poff + 56:poff + 88], dtype=np.int64)
        assert list(rec) == [9, 9, 9, 16]
    bad = make_problems([9], pitch=8)
    assert lib.ps_batch_table_fill_ex(host, nbytes, bad, 1, _lib.PS_F64, 0, 0, 0, 0, None) == _lib.PS_ERR_ARG
    assert b"pitch" in lib.ps_last_error()
    for flags, dtype in ((_lib.PS_BATCH_COLUMN | _lib.PS_BATCH_ZMARCH, _lib.PS_F64), (64, _lib.PS_F64),
                         (_lib.PS_BATCH_CI_SCALED, _lib.PS_F32),
                         (_lib.PS_BATCH_CI_SCALED | _lib.PS_BATCH_COLUMN, _lib.PS_F64)):
        assert lib.ps_batch_table_fill_ex(host, nbytes, arr, 2, dtype, 0, 0, 0, flags, None) == _lib.PS_ERR_ARG
    assert lib.ps_batch_table_kernel(None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_step_ex(0x1000, None, 0, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_run_ex(0x1000, None, 4, 0, None) == _lib.PS_ERR_ARG
    if not have_driver(lib):
        assert lib.ps_batch_table_kernel(host) == 0
        st = lib.ps_batch_table_fill_ex(host, nbytes, arr, 2, _lib.PS_F64, 0, 0, 0, _lib.PS_BATCH_ZMARCH, None)
        assert st == _lib.PS_ERR_UNSUPPORTED and b"encoder" in lib.ps_last_error()


def test_adjoint2_and_batch_pair_calls_reject_bad_arguments(lib):
    """The fused transposed pair and the batched pair calls check their arguments on
    the host before any launch."""
    D, E, F = 0x290000000, 0x390000000, 0x490000000
    f32, f64 = _lib.PS_F32, _lib.PS_F64

    def adj2(Tbar=E, Cib=F, yb=A, T1=B, T0=C, Ci=D, dtype=f32, flags=0, n=(8, 8, 8)):
        return lib.ps_diffusion3d_adjoint2_ex(Tbar, Cib, yb, T1, T0, Ci, 1.0, 1e-3, 7.0, 7.0, 7.0, *n, dtype,
                                              flags, None)
    assert adj2(flags=1) == _lib.PS_ERR_ARG
    assert adj2(T0=None) == _lib.PS_ERR_ARG
    assert adj2(Tbar=A) == _lib.PS_ERR_ALIAS      # Tbar is ybar
    assert adj2(Tbar=C) == _lib.PS_ERR_ALIAS      # Tbar is the second state
    assert adj2(Cib=B) == _lib.PS_ERR_ALIAS       # Cibar is the first state
    assert adj2(dtype=f64) == _lib.PS_ERR_UNSUPPORTED
    assert adj2(n=(6, 8, 8)) == _lib.PS_ERR_UNSUPPORTED  # rows of 24 bytes
    assert b"16" in lib.ps_last_error()
    assert lib.ps_diffusion3d_batch_step2_ex(0x1000, None, 0, None) == _lib.PS_ERR_ARG
    # a column-march table has no pair list; run_ex refuses PS_RUN_TEMPORAL2 on it
    arr = make_problems([9, 12])
    nbytes = lib.ps_batch_table_bytes_ex(arr, 2, f64, 0, 0, 0, _lib.PS_BATCH_COLUMN)
    buf = (ctypes.c_char * (nbytes + 64))()
    off = (-ctypes.addressof(buf)) % 64
    host = (ctypes.c_char * nbytes).from_buffer(buf, off)
    assert lib.ps_batch_table_fill_ex(host, nbytes, arr, 2, f64, 0, 0, 0, _lib.PS_BATCH_COLUMN, None) == _lib.PS_OK
    assert lib.ps_diffusion3d_batch_run_ex(0x1000, host, 4, _lib.PS_RUN_TEMPORAL2, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_step2_ex(0x1000, host, 0, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_step_ex(0x1000, host, 2, None) == _lib.PS_ERR_ARG  # parity
    # pair tables: FP64 needs the pre-scaled coefficient; the column march has no pairs
    for flags, dtype in ((_lib.PS_BATCH_TEMPORAL2, f64), (_lib.PS_BATCH_TEMPORAL2 | _lib.PS_BATCH_COLUMN, f32)):
        assert lib.ps_batch_table_fill_ex(host, nbytes, arr, 2, dtype, 0, 0, 0, flags, None) == _lib.PS_ERR_ARG


def test_diffusion2d_rejects_bad_arguments(lib):
    f64, f32 = _lib.PS_F64, _lib.PS_F32

    def step2d(T2=B, T=A, Ci=C, nx=8, ny=8, dtype=f64, flags=0, dx=7.0, dy=7.0):
        return lib.ps_diffusion2d_step(T2, T, Ci, 1.0, 1e-3, dx, dy, nx, ny, dtype, flags, None)
    assert step2d(nx=2) == _lib.PS_ERR_ARG
    assert step2d(T=None) == _lib.PS_ERR_ARG
    assert step2d(T2=A) == _lib.PS_ERR_ALIAS
    assert step2d(T=A + 8) == _lib.PS_ERR_ALIGN
    assert step2d(flags=_lib.PS_RUN_GRAPH) == _lib.PS_ERR_ARG  # run only
    assert step2d(flags=_lib.PS_RUN_CI_SCALED, dtype=f32) == _lib.PS_ERR_UNSUPPORTED
    assert step2d(flags=_lib.PS_RUN_CI_SCALED, dy=6.0) == _lib.PS_ERR_UNSUPPORTED
    odd = ctypes.c_int(-1)
    assert lib.ps_diffusion2d_run(A, B, C, 1.0, 1e-3, 7.0, 7.0, 8, 8, -1, f64, 0, None,
                                  ctypes.byref(odd)) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion2d_run(A, B, C, 1.0, 1e-3, 7.0, 7.0, 8, 8, 3, f64, 0x40, None,
                                  ctypes.byref(odd)) == _lib.PS_ERR_ARG
    dt = ctypes.c_double(0.0)
    assert lib.ps_diffusion2d_stable_dt(None, C, 8, 8, 1.0, 1.0, 1.0, f64, A, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion2d_stable_dt(ctypes.byref(dt), C, 2, 8, 1.0, 1.0, 1.0, f64, A, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion2d_stable_dt(ctypes.byref(dt), None, 8, 8, 1.0, 1.0, 1.0, f64, A, None) == _lib.PS_ERR_ARG
    assert lib.ps_diffusion2d_stable_dt(ctypes.byref(dt), C, 8, 8, float("nan"), 1.0, 1.0, f64, A,
                                        None) == _lib.PS_ERR_ARG


def test_launch_overrides_set_get_and_range(lib):
    """The launch-shape overrides: every PS_OVERRIDE_* value reads back, out-of-range
    keys and values are rejected, 0 restores the library's own choice."""
    v = ctypes.c_int(-1)
    for name, which in _lib.PS_OVERRIDE.items():
        assert lib.ps_get_launch_override(which, ctypes.byref(v)) == _lib.PS_OK and v.value == 0
        value = 1 if name in ("adj_plain", "f64_px2", "step_plain") else 17
        assert lib.ps_set_launch_override(which, value) == _lib.PS_OK
        assert lib.ps_get_launch_override(which, ctypes.byref(v)) == _lib.PS_OK and v.value == value
        assert lib.ps_set_launch_override(which, 0) == _lib.PS_OK
    assert lib.ps_set_launch_override(len(_lib.PS_OVERRIDE), 1) == _lib.PS_ERR_ARG
    assert lib.ps_set_launch_override(-1, 1) == _lib.PS_ERR_ARG
    assert lib.ps_set_launch_override(_lib.PS_OVERRIDE["adj_plain"], 2) == _lib.PS_ERR_ARG
    assert lib.ps_set_launch_override(_lib.PS_OVERRIDE["kchunk"], 4097) == _lib.PS_ERR_ARG
    assert lib.ps_set_launch_override(_lib.PS_OVERRIDE["kchunk"], -3) == _lib.PS_ERR_ARG
    assert lib.ps_get_launch_override(0, None) == _lib.PS_ERR_ARG


def test_dot_static_rejects_bad_arguments(lib):
    """The no-allocation dot product: null pointers, element misalignment, n < 1 and
    n beyond the static capacity are refused before any launch or device call."""
    f64, f32 = _lib.PS_F64, _lib.PS_F32
    assert lib.ps_dot_static(None, A, B, 8, f64, None) == _lib.PS_ERR_ARG
    assert lib.ps_dot_static(C, None, B, 8, f64, None) == _lib.PS_ERR_ARG
    assert lib.ps_dot_static(C, A, B, 8, 7, None) == _lib.PS_ERR_ARG
    assert lib.ps_dot_static(C, A + 4, B, 8, f64, None) == _lib.PS_ERR_ALIGN
    assert lib.ps_dot_static(C, A, B + 2, 8, f32, None) == _lib.PS_ERR_ALIGN
    assert lib.ps_dot_static(C, A, B, 0, f64, None) == _lib.PS_ERR_ARG
    assert lib.ps_dot_static(C, A, B, 4096 * 32768 + 1, f64, None) == _lib.PS_ERR_UNSUPPORTED
