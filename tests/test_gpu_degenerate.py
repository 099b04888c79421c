"""Degenerate inputs of the step, on every FP64 kernel form and on FP32:

* no diffusion - Ci = 0, or dt = 0 - leaves the field unchanged, and a zero field
  stays zero;
* fields at the bottom of the FP64 range: normal values near 2^-1020 whose
  neighbour differences, and so the packed Laplacian, are subnormal (gradual
  underflow, as the oracle's IEEE arithmetic has it), of either sign, and a field of
  mixed signs around zero there (the general path with its smallest scales);
* NaN and Inf at interior nodes spread exactly as in the oracle's evaluation: the
  same nodes end NaN, the same end Inf, and the finite ones agree within 1e-12;
* a field at the top of the range whose Laplacian overflows goes to +-Inf (then NaN)
  where the oracle's does.

The FP64 forms: the pre-scaled step with four and with two nodes per thread, the
column kernel (odd nx), Ci as given on equal spacings (one pack and a DMUL) and on
unequal spacings (K*S products), and fused step pairs; the transposed step on the
pre-scaled coefficient near underflow too."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

U32 = 2.0 ** -24
FP64_FORMS = {  # name: (shape nx, ny, nz; equal spacings?; pre-scaled?; fused pairs?)
    "scaled4": ((68, 21, 13), True, True, False),
    "scaled2": ((66, 21, 13), True, True, False),
    "column": ((67, 21, 13), True, True, False),
    "as_given_iso": ((68, 21, 13), True, False, False),
    "as_given_aniso": ((68, 21, 13), False, False, False),
    "pairs": ((68, 21, 13), True, True, True),
}


def grid(form):
    (nx, ny, nz), equal, _, _ = FP64_FORMS[form]
    if equal:
        d = 1.0 / (max(nx, ny, nz) - 1)
        return (nx, ny, nz), (1.0 / d,) * 3, d * d
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    return (nx, ny, nz), inputs.inverse_spacing(nx, ny, nz), min(dx * dx, dy * dy, dz * dz)


def run64(form, T0, Ci, lam, dt, inv, nt):
    _, _, scaled, pairs = FP64_FORMS[form]
    T = to_dev(T0)
    C = to_dev(Ci)
    if scaled:
        C = api.scale_ci(C, lam, dt, inv)
    res = api.run(T, torch.empty_like(T), C, lam, dt, inv, nt, ci_scaled=scaled, temporal2=pairs)
    assert api.device_error() == 0
    return to_host(res)


def same(a, b):
    """Equal values (a signed zero may come out with either sign)."""
    return np.array_equal(a, b)


@pytest.mark.parametrize("form", list(FP64_FORMS))
def test_fp64_no_diffusion_and_zero_field(form):
    (nx, ny, nz), inv, d2 = grid(form)
    T0 = 1.7 + inputs.random_field((nz, ny, nx), 5, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d2 / Ci.max() / 6.1
    assert same(run64(form, T0, np.zeros_like(Ci), 1.0, dt, inv, 4), T0)   # Ci = 0
    assert same(run64(form, T0, Ci, 1.0, 0.0, inv, 4), T0)                 # dt = 0
    Z = np.zeros_like(T0)
    assert same(run64(form, Z, Ci, 1.0, dt, inv, 4), Z)                    # zero field


def test_fp32_no_diffusion_and_zero_field():
    nx, ny, nz = 68, 21, 13
    D0 = inputs.random_field((nz, ny, nx), 5, -1.0, 1.0).astype(np.float32)
    Ci = inputs.ci_random(nx, ny, nz).astype(np.float32)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / float(Ci.max()) / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    for D, C, step_dt in ((D0, np.zeros_like(Ci), dt), (D0, Ci, 0.0), (np.zeros_like(D0), Ci, dt)):
        Dd = torch.from_numpy(D).cuda()
        res = api.run(Dd, torch.empty_like(Dd), torch.from_numpy(C).cuda(), 1.0, step_dt, inv, 4)
        assert np.array_equal(res.cpu().numpy(), D)
        # the compensated two-float step from a zero correction: the same
        comp = api.compensation_fields(Dd)
        Dd = torch.from_numpy(D).cuda()
        res = api.run(Dd, torch.empty_like(Dd), torch.from_numpy(C).cuda(), 1.0, step_dt, inv, 4, comp=comp)
        assert np.array_equal(res.cpu().numpy(), D)
        assert not torch.any(comp[0] != 0) and not torch.any(comp[1] != 0)
    assert api.device_error() == 0


def tiny_field(kind, shape):
    nx, ny, nz = shape
    u = inputs.random_field((nz, ny, nx), 23, 0.0, 1.0)
    if kind == "positive":   # normal values just above the normal range, subnormal differences
        return 2.0 ** -1020 * (1.0 + u)
    if kind == "negative":
        return -(2.0 ** -1020) * (1.0 + u)
    if kind == "mixed":      # both signs, zeros, subnormal and normal values around 2^-1022
        T = 2.0 ** -1021 * (2.0 * u - 1.0)
        T[::4, ::3, ::5] = 0.0
        return T
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["positive", "negative", "mixed"])
@pytest.mark.parametrize("form", list(FP64_FORMS))
def test_fp64_near_underflow_matches_oracle(form, kind):
    (nx, ny, nz), inv, d2 = grid(form)
    T0 = tiny_field(kind, (nx, ny, nz))
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d2 / Ci.max() / 6.1
    nt = 4
    ref = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
    got = run64(form, T0, Ci, 1.0, dt, inv, nt)
    # the update is a good fraction of each value here: dropping it would miss by ~1e-2
    assert np.max(np.abs(ref - T0)) > 1e-3 * np.max(np.abs(T0))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(T0))


@pytest.mark.parametrize("kind", ["positive", "mixed"])
def test_fp64_transposed_step_near_underflow(kind):
    """dL/dCs accumulates ybar * L(T) with L(T) subnormal (packed like the step's)."""
    (nx, ny, nz), inv, d2 = grid("scaled4")
    T = tiny_field(kind, (nx, ny, nz))
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d2 / Ci.max() / 6.1
    ybar = inputs.random_field((nz, ny, nx), 31, -1.0, 1.0)
    cib_ref = np.zeros_like(T)
    tbar_ref = oracle.adjoint_step(ybar, T, Ci, cib_ref, 1.0, dt, *inv)
    Cs = api.scale_ci(to_dev(Ci), 1.0, dt, inv)
    tbar, csbar = torch.empty_like(Cs), torch.zeros_like(Cs)
    api.adjoint(tbar, csbar, to_dev(ybar), to_dev(T), Cs, 1.0, dt, inv, ci_scaled=True)
    cib = to_host(api.scale_ci(csbar, 1.0, dt, inv))  # dL/dCi = dt*lam*_dx^2 * dL/dCs
    assert rel_linf(to_host(tbar), tbar_ref) <= 1e-14
    assert np.max(np.abs(cib - cib_ref)) <= 1e-12 * np.max(np.abs(cib_ref))
    assert np.max(np.abs(cib_ref)) > 0.0
    assert api.device_error() == 0


def nonfinite_field(shape):
    nx, ny, nz = shape
    T = 1.7 + inputs.random_field((nz, ny, nx), 41, 0.0, 1.0)
    T[5, 9, 20] = np.nan
    T[8, 4, 50] = np.inf
    return T


def check_nonfinite(got, ref, scale, tol):
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(np.isposinf(got), np.isposinf(ref))
    assert np.array_equal(np.isneginf(got), np.isneginf(ref))
    fin = np.isfinite(ref)
    assert np.max(np.abs(got[fin] - ref[fin])) <= tol * scale


@pytest.mark.parametrize("nt", [1, 3])
@pytest.mark.parametrize("form", list(FP64_FORMS))
def test_fp64_nan_and_inf_spread_like_the_oracle(form, nt):
    (nx, ny, nz), inv, d2 = grid(form)
    T0 = nonfinite_field((nx, ny, nz))
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d2 / Ci.max() / 6.1
    ref = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
    assert np.isnan(ref).sum() > 1 and np.isinf(ref).sum() > 1
    check_nonfinite(run64(form, T0, Ci, 1.0, dt, inv, nt), ref, 2.7, 1e-12)


@pytest.mark.parametrize("nt", [1, 3])
def test_fp32_nan_and_inf_spread_like_the_oracle(nt):
    nx, ny, nz = 68, 21, 13
    D0 = (nonfinite_field((nx, ny, nz)) - 1.7).astype(np.float32)
    Ci = inputs.ci_random(nx, ny, nz).astype(np.float32)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / float(Ci.max()) / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    D = torch.from_numpy(D0).cuda()
    got = api.run(D, torch.empty_like(D), torch.from_numpy(Ci).cuda(), 1.0, dt, inv, nt).double().cpu().numpy()
    ref = oracle.run(D0.astype(np.float64), Ci.astype(np.float64), 1.0, dt, *inv, nt)
    check_nonfinite(got, ref, 1.0, nt * 13 * U32)
    assert api.device_error() == 0


@pytest.mark.parametrize("form", ["scaled4", "scaled2", "column", "pairs"])
def test_fp64_overflowing_laplacian_gives_inf_like_the_oracle(form):
    """A checkerboard of 2^1023 and 1.9 * 2^1023 (one binade): the sum of the neighbours
    minus six centres is about +-5.4 * 2^1023, past the largest double, so the interior
    goes to +-Inf as in the oracle (whose scaled second differences overflow) - not to
    a wrapped bit pattern - and the next step to NaN, again as in the oracle."""
    (nx, ny, nz), inv, d2 = grid(form)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    T0 = np.where((i + j + k) % 2 == 0, 1.0, 1.9) * 2.0 ** 1023
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d2 / Ci.max() / 6.1
    for nt in (1, 2):
        ref = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
        inner = ref[1:-1, 1:-1, 1:-1]
        assert np.all(np.isinf(inner)) if nt == 1 else np.all(np.isnan(inner))
        check_nonfinite(run64(form, T0, Ci, 1.0, dt, inv, nt), ref, 2.0 ** 1023, 1e-12)


ADJ_FORMS = {  # name: (pre-scaled coefficient?, dtype)
    "scaled": (True, torch.float64),
    "as_given": (False, torch.float64),
    "f32": (False, torch.float32),
}


def adjoint_case(form, nx=68, ny=21, nz=13):
    scaled, dtype = ADJ_FORMS[form]
    d = 1.0 / (max(nx, ny, nz) - 1)
    inv = (1.0 / d,) * 3
    T = 1.7 + inputs.random_field((nz, ny, nx), 51, 0.0, 1.0)
    if dtype == torch.float32:
        T = T - 1.7
    Ci = inputs.ci_random(nx, ny, nz)
    dt = d * d / Ci.max() / 6.1
    ybar = inputs.random_field((nz, ny, nx), 52, -1.0, 1.0)
    return scaled, dtype, inv, T, Ci, dt, ybar


def gpu_adjoint(scaled, dtype, inv, T, Ci, dt, ybar, cib0):
    Td, Cd, Yd = to_dev(T, dtype), to_dev(Ci, dtype), to_dev(ybar, dtype)
    C = api.scale_ci(Cd, 1.0, dt, inv) if scaled else Cd
    tbar, cib = torch.empty_like(Td), to_dev(cib0, dtype)
    api.adjoint(tbar, cib, Yd, Td, C, 1.0, dt, inv, ci_scaled=scaled)
    assert api.device_error() == 0
    return to_host(tbar), to_host(cib)


@pytest.mark.parametrize("form", list(ADJ_FORMS))
def test_transposed_step_degenerate_inputs(form):
    """Zero cotangent: Tbar = 0 and the coefficient gradient unchanged.  Zero coefficient
    (Ci = 0): w = 0, so Tbar = ybar exactly.  dt = 0 (coefficient as given): Tbar = ybar
    and the coefficient gradient unchanged, bit for bit."""
    scaled, dtype, inv, T, Ci, dt, ybar = adjoint_case(form)
    cib0 = inputs.random_field(T.shape, 53, -1.0, 1.0)
    if dtype == torch.float32:
        cib0 = cib0.astype(np.float32).astype(np.float64)
        ybar = ybar.astype(np.float32).astype(np.float64)
    tb, cb = gpu_adjoint(scaled, dtype, inv, T, Ci, dt, np.zeros_like(ybar), cib0)
    assert not np.any(tb) and np.array_equal(cb, cib0)
    tb, _ = gpu_adjoint(scaled, dtype, inv, T, np.zeros_like(Ci), dt, ybar, cib0)
    assert np.array_equal(tb, ybar)
    if not scaled:  # the pre-scaled form needs dt > 0 to form Cs = dt*lam*_dx^2*Ci
        tb, cb = gpu_adjoint(scaled, dtype, inv, T, Ci, 0.0, ybar, cib0)
        assert np.array_equal(tb, ybar) and np.array_equal(cb, cib0)


@pytest.mark.parametrize("form", list(ADJ_FORMS))
def test_transposed_step_nonfinite_cotangent(form):
    """NaN and Inf in ybar: every node the oracle's transposed step makes non-finite is
    non-finite on the GPU too, and every node the GPU leaves finite agrees with the oracle.
    (The FP64 forms hold w in fixed point at a scale shared by a CTA's march; a non-finite
    w marks that CTA's Tbar NaN, a superset of the oracle's non-finite nodes.)"""
    scaled, dtype, inv, T, Ci, dt, ybar = adjoint_case(form)
    ybar[5, 9, 20] = np.nan
    ybar[8, 4, 50] = np.inf
    if dtype == torch.float32:
        ybar = ybar.astype(np.float32).astype(np.float64)
        T = T.astype(np.float32).astype(np.float64)
        Ci = Ci.astype(np.float32).astype(np.float64)
    cib0 = np.zeros_like(T)
    tb, cb = gpu_adjoint(scaled, dtype, inv, T, Ci, dt, ybar, cib0)
    cib_ref = np.zeros_like(T)
    tb_ref = oracle.adjoint_step(ybar, T, Ci, cib_ref, 1.0, dt, *inv)
    if scaled:  # the GPU accumulated dL/dCs; dL/dCi = dt*lam*_dx^2 * dL/dCs
        cb = cb * (dt * inv[0] * inv[0])
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    for got, ref in ((tb, tb_ref), (cb, cib_ref)):
        assert np.all(~np.isfinite(got[~np.isfinite(ref)]))
        fin = np.isfinite(got)
        assert np.all(np.isfinite(ref[fin]))
        scale = np.max(np.abs(ref[np.isfinite(ref)]))
        assert np.max(np.abs(got[fin] - ref[fin])) <= tol * scale
        assert fin.sum() > 0.5 * got.size  # the NaN stays local to the CTAs that met it
