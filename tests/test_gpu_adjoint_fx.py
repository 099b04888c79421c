"""The reverse sweep with dL/dT held as an int64 field at one scale (ps_adjoint_fx_*,
api.FixedPointSweep) against the FP64 oracle's adjoint of the plain step, step by step
and over sweeps, including the steps that rescale the field by a power of two when its
largest value leaves [2^50, 2^60), and the flag for coefficients it cannot take.

Csbar accumulates dL/dCs = ybar * L(T); K * Csbar (K = dt*lam*_d^2) is compared with
the oracle's Cibar term."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import _lib, api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def iso_fields(nx, ny, nz, seed=3):
    T = 1.7 + inputs.random_field((nz, ny, nx), seed, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    lam = 1.0
    d = 1.0 / (max(nx, ny, nz) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T, Ci, lam, dt, (1.0 / d,) * 3


def fx_sweep(ybar, states, Cs, csbar0=None):
    """GPU fixed-point sweep over the states (applied last to first); returns
    (dL/dT, Csbar) on the host."""
    Csb = to_dev(csbar0) if csbar0 is not None else torch.zeros(ybar.shape, dtype=torch.float64,
                                                                device="cuda")
    sw = api.FixedPointSweep(Csb)
    sw.start(to_dev(ybar))
    for T in reversed(states):
        sw.step(Csb, to_dev(T), Cs)
    return to_host(sw.finish()), to_host(Csb)


SHAPES = [(4, 5, 6), (6, 7, 5), (64, 8, 9), (66, 19, 20), (130, 67, 33), (132, 21, 17), (256, 35, 19)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fx_step_matches_oracle(shape):
    T, Ci, lam, dt, inv = iso_fields(*shape)
    K = dt * lam * inv[0] * inv[0]
    ybar = inputs.random_field(T.shape, 5)
    cib = np.zeros_like(T)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    tbar, csb = fx_sweep(ybar, [T], Cs)
    assert rel_linf(tbar, ref) <= 1e-14
    assert np.max(np.abs(K * csb - cib)) <= 1e-14 * np.max(np.abs(cib))
    assert api.device_error() == 0


@pytest.mark.parametrize("shape,nt", [((66, 19, 20), 9), ((132, 21, 17), 14)])
def test_fx_sweep_matches_oracle_gradient(shape, nt):
    """nt transposed steps over the states of a forward run: dL/dT0 and dL/dCi of
    L = 1/2||T(nt) - T_obs||^2 against the oracle's gradient."""
    T0, Ci, lam, dt, inv = iso_fields(*shape)
    Tobs = oracle.run(T0, Ci * 1.1, lam, dt, *inv, nt)
    L_ref, dT0_ref, dCi_ref = oracle.gradient(T0, Ci, Tobs, lam, dt, *inv, nt)
    states = [T0]
    for _ in range(nt - 1):
        states.append(oracle.run(states[-1], Ci, lam, dt, *inv, 1))
    resid = oracle.run(T0, Ci, lam, dt, *inv, nt) - Tobs
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    K = dt * lam * inv[0] * inv[0]
    dT0, csb = fx_sweep(resid, states, Cs)
    assert rel_linf(dT0, dT0_ref) <= 1e-12
    assert rel_linf(K * csb, dCi_ref) <= 1e-12


def test_fx_equals_fp64_sweep_closely():
    """The fixed-point sweep and the FP64 transposed step (api.adjoint, pre-scaled)
    give the same dL/dT0 and dL/dCs to a few units in the last place of the largest."""
    T, Ci, lam, dt, inv = iso_fields(130, 67, 33)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    ybar = inputs.random_field(T.shape, 9)
    states = [T + 0.01 * k * inputs.random_field(T.shape, 20 + k) for k in range(12)]
    a_tbar, a_csb = fx_sweep(ybar, states, Cs)
    yb = to_dev(ybar)
    tb = torch.empty_like(yb)
    csb = torch.zeros_like(yb)
    for S in reversed(states):
        api.adjoint(tb, csb, yb, to_dev(S), Cs, lam, dt, inv, ci_scaled=True)
        yb, tb = tb, yb
    assert rel_linf(a_tbar, to_host(yb)) <= 1e-14
    assert rel_linf(a_csb, to_host(csb)) <= 1e-14


def fp64_sweep(ybar, states, Cs):
    yb = to_dev(ybar)
    tb = torch.empty_like(yb)
    csb = torch.zeros_like(yb)
    for S in reversed(states):
        api.adjoint(tb, csb, yb, to_dev(S), Cs, 1.0, 1.0, (1.0, 1.0, 1.0), ci_scaled=True)
        yb, tb = tb, yb
    return to_host(yb), to_host(csb)


def test_fx_rescales_a_decaying_field():
    """A spike at the centre of a 64^3 grid spreads under Cs = 1/6.1: after 40
    transposed steps its largest value has fallen by more than 2^8, below the window
    [2^50, 2^60) the sweep keeps, so the field is rescaled upwards on the way; the
    result matches the FP64 sweep relative to its own largest value."""
    n = 64
    ybar = np.zeros((n, n, n))
    ybar[32, 32, 32] = 1.0
    ybar[20, 33, 40] = -0.5
    Cs = torch.full((n, n, n), 1.0 / 6.1, dtype=torch.float64, device="cuda")
    states = [1.7 + inputs.random_field((n, n, n), 6, 0.0, 1.0)] * 40
    a_tbar, a_csb = fx_sweep(ybar, states, Cs)
    ref, ref_csb = fp64_sweep(ybar, states, Cs)
    assert np.max(np.abs(ref)) < 2.0 ** -8 * np.max(np.abs(ybar))  # decayed past the window
    assert rel_linf(a_tbar, ref) <= 1e-13
    assert rel_linf(a_csb, ref_csb) <= 1e-13


def test_fx_rescales_a_growing_field():
    """With Cs = 0.24 (not a stable step, but inside the |Cs| < 1/4 the sweep takes)
    the checkerboard grows by about 1.9 per transposed step: the largest value leaves
    [2^50, 2^60) again and again and is rescaled downwards each time."""
    nx, ny, nz = 64, 20, 18
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ybar = np.where((i + j + k) % 2 == 0, 1.0, -1.0) * (1.0 + 0.1 * inputs.random_field((nz, ny, nx), 5, 0.0, 1.0))
    Cs = torch.full((nz, ny, nx), 0.24, dtype=torch.float64, device="cuda")
    states = [1.7 + inputs.random_field((nz, ny, nx), 7, 0.0, 1.0)] * 12
    a_tbar, a_csb = fx_sweep(ybar, states, Cs)
    ref, ref_csb = fp64_sweep(ybar, states, Cs)
    assert np.max(np.abs(ref)) > 64.0 * np.max(np.abs(ybar))  # grew past the window, several times
    assert rel_linf(a_tbar, ref) <= 1e-13
    assert rel_linf(a_csb, ref_csb) <= 1e-13


@pytest.mark.parametrize("bad", ["large", "nan"])
def test_fx_flags_coefficients_it_cannot_take(bad):
    """|Cs| >= 1/4 at an interior node, or a NaN, marks the sweep bad: its result is NaN."""
    T, Ci, lam, dt, inv = iso_fields(64, 12, 10)
    Cs_h = Ci * dt * inv[0] ** 2
    Cs_h[5, 6, 7] = 0.3 if bad == "large" else np.nan
    tbar, _ = fx_sweep(inputs.random_field(T.shape, 5), [T, T], to_dev(Cs_h))
    assert np.all(np.isnan(tbar))


def test_fx_rejects_bad_arguments_and_odd_rows():
    lib = _lib.load()
    T = torch.zeros((6, 5, 7), dtype=torch.float64, device="cuda")  # nx*8 not a multiple of 16
    Y = torch.zeros(T.shape, dtype=torch.int64, device="cuda")
    st = torch.zeros(lib.ps_adjoint_fx_state_bytes(), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.ps_diffusion3d_adjoint_fx(Y.clone().data_ptr(), T.clone().data_ptr(), Y.data_ptr(), T.data_ptr(),
                                         T.clone().data_ptr(), 7, 5, 6, st.data_ptr(), 0, s) == \
        _lib.PS_ERR_UNSUPPORTED
    assert not api.FixedPointSweep.supported(T)
    assert lib.ps_diffusion3d_adjoint_fx(Y.data_ptr(), T.data_ptr(), Y.data_ptr(), T.data_ptr(),
                                         T.data_ptr(), 7, 5, 6, st.data_ptr(), 0, s) == _lib.PS_ERR_ALIAS
    assert lib.ps_adjoint_fx_end(T.data_ptr(), Y.data_ptr(), T.numel(), st.data_ptr(), -1, s) == _lib.PS_ERR_ARG
