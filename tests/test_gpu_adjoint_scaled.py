"""Transposed step on the pre-scaled coefficient Cs = dt*lam*_d^2*Ci (FP64, equal
spacings) against the FP64 oracle's adjoint of the plain step.

The pre-scaled adjoint returns Tbar (the same quantity as the plain adjoint) and
accumulates dL/dCs = ybar * L(T); dL/dCi = K * dL/dCs with K = dt*lam*_d^2, so
K * Csbar is compared with the oracle's Cibar term."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs
from paper_2211_15634_gb300 import autograd as ag

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def iso_fields(nx, ny, nz, seed=3):
    """State, coefficient and spacing of a grid with one spacing d on every axis."""
    T = 1.7 + inputs.random_field((nz, ny, nx), seed, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    lam = 1.0
    d = 1.0 / (max(nx, ny, nz) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T, Ci, lam, dt, (1.0 / d,) * 3


def scaled_adjoint(ybar, T, Ci, lam, dt, inv, csbar0=None):
    """GPU pre-scaled adjoint; returns (Tbar, K * Csbar) on the host."""
    K = dt * lam * inv[0] * inv[0]
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    Tbar = torch.empty(T.shape, dtype=torch.float64, device="cuda")
    Csb = to_dev(csbar0) if csbar0 is not None else torch.zeros_like(Tbar)
    api.adjoint(Tbar, Csb, to_dev(ybar), to_dev(T), Cs, lam, dt, inv, ci_scaled=True)
    return to_host(Tbar), K * to_host(Csb)


SHAPES = [(3, 3, 3), (4, 5, 6), (5, 6, 7), (37, 29, 23), (64, 8, 9), (66, 19, 20), (130, 67, 33),
          (132, 21, 17), (256, 35, 19)]


@pytest.mark.parametrize("shape", SHAPES)
def test_scaled_adjoint_step_matches_oracle(shape):
    T, Ci, lam, dt, inv = iso_fields(*shape)
    ybar = inputs.random_field(T.shape, 5)
    cib = np.zeros_like(T)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    Tbar, cig = scaled_adjoint(ybar, T, Ci, lam, dt, inv)
    assert rel_linf(Tbar, ref) <= 1e-14
    assert np.max(np.abs(cig - cib)) <= 1e-14 * np.max(np.abs(cib))
    assert api.device_error() == 0


def test_scaled_adjoint_accumulates_into_csbar():
    nx, ny, nz = 68, 20, 15
    T, Ci, lam, dt, inv = iso_fields(nx, ny, nz)
    K = dt * lam * inv[0] * inv[0]
    ybar = inputs.random_field(T.shape, 5)
    cib0 = inputs.random_field(T.shape, 6)
    cib = cib0.copy()
    oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    _, cig = scaled_adjoint(ybar, T, Ci, lam, dt, inv, csbar0=cib0 / K)
    inner = np.zeros(T.shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.max(np.abs(cig - cib)) <= 1e-14 * np.max(np.abs(cib))
    # boundary entries are left as they were
    assert np.array_equal(cig[~inner], K * (cib0 / K)[~inner])


@pytest.mark.parametrize("kchunk", ["0", "1", "3", "40"])
def test_scaled_adjoint_scale_growth(launch_override, kchunk):
    """ybar growing by 10^4 along z (with sign changes and exact zeros): the CTA's
    fixed-point scale grows in mid-march, so tiles and registers already held are
    shifted; every plane still matches the oracle at its own magnitude."""
    launch_override(adj_kchunk=kchunk)
    nx, ny, nz = 68, 21, 40
    T, Ci, lam, dt, inv = iso_fields(nx, ny, nz)
    ybar = inputs.random_field(T.shape, 5) * (10.0 ** (np.arange(nz) / 10.0))[:, None, None]
    ybar[:, ::4, ::3] = 0.0
    cib = np.zeros_like(T)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    Tbar, cig = scaled_adjoint(ybar, T, Ci, lam, dt, inv)
    for k in range(nz):
        assert np.max(np.abs(Tbar[k] - ref[k])) <= 1e-13 * np.max(np.abs(ref[k])), k
        if 1 <= k <= nz - 2:
            assert np.max(np.abs(cig[k] - cib[k])) <= 1e-13 * np.max(np.abs(cib[k])), k
    assert api.device_error() == 0


def test_scaled_adjoint_general_laplacian_path():
    """States that change sign and binade at every node send the T-Laplacian of the
    Csbar term through the fixed-point general path."""
    nx, ny, nz = 66, 31, 17
    _, Ci, lam, dt, inv = iso_fields(nx, ny, nz)
    T = inputs.random_field((nz, ny, nx), 77, -1.0, 1.0)
    T[::3, :, ::5] = 0.0
    T[1::4, ::2, :] *= 1e-9
    ybar = inputs.random_field(T.shape, 5)
    cib = np.zeros_like(T)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    Tbar, cig = scaled_adjoint(ybar, T, Ci, lam, dt, inv)
    assert rel_linf(Tbar, ref) <= 1e-14
    assert np.max(np.abs(cig - cib)) <= 1e-14 * np.max(np.abs(cib))


def iso_inverse_problem(nx, ny, nz, nt):
    """The inverse problem of the gradient tests on a grid with equal spacings."""
    lam = 1.0
    T0 = inputs.t0_gaussian(nx, ny, nz)
    Ci_true = inputs.ci_smooth(nx, ny, nz)
    Ci = inputs.ci_constant(nx, ny, nz) + 0.02 * inputs.random_field((nz, ny, nx), 8)
    d = 1.0 / (max(nx, ny, nz) - 1)
    dt = d * d / lam / (1.5 / inputs.C0) / 6.1
    inv = (1.0 / d,) * 3
    Tobs = oracle.run(T0, Ci_true, lam, dt, *inv, nt)
    return T0, Ci, Tobs, lam, dt, inv


@pytest.mark.parametrize("shape,nt", [((20, 20, 20), 12), ((33, 17, 21), 9), ((68, 40, 30), 16)])
def test_scaled_gradient_matches_oracle(shape, nt):
    T0, Ci, Tobs, lam, dt, inv = iso_inverse_problem(*shape, nt)
    L_ref, dT0_ref, dCi_ref = oracle.gradient(T0, Ci, Tobs, lam, dt, *inv, nt)
    C = to_dev(Ci)
    assert ag.coefficient(C, lam, dt, inv)[1]  # the pre-scaled path is taken
    L, dT0, dCi = ag.loss_and_grad(to_dev(T0), C, to_dev(Tobs), lam, dt, inv, nt)
    assert abs(float(L) - L_ref) <= 1e-12 * L_ref
    assert rel_linf(to_host(dT0), dT0_ref) <= 1e-10
    assert rel_linf(to_host(dCi), dCi_ref) <= 1e-10


@pytest.mark.parametrize("every", [1, 3, 13])
def test_scaled_checkpoint_interval_does_not_change_gradient(every):
    nx, ny, nz, nt = 24, 14, 18, 13
    T0, Ci, Tobs, lam, dt, inv = iso_inverse_problem(nx, ny, nz, nt)
    base = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt, every=nt)
    got = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt, every=every)
    for a, b in zip(base, got):
        assert torch.equal(a, b)
