"""Pins of the oracle's explicit-notation step (the solver the paper's Results set beside
Fig. 1's: the stencil written out on indices, second differences A[i+1] - 2*A[i] + A[i-1]).

The same facts pin it as pin Fig. 1's form - the constant field, the discrete sine
eigenmode's exact decay factor, the dense Kronecker matrix on tiny grids - each an
independent formulation; and the two notations agree to rounding (a few units in the
last place per step), since they are one operator.  CPU only.
"""
import numpy as np
import pytest

from paper_2211_15634_gb300 import inputs
from test_oracle_pins import LAM, dense_step_matrix, interior_mask, rel_linf, small_problem


def test_constant_field_stays_bitwise(oracle_mod):
    nx, ny, nz = 11, 9, 7
    T0 = np.full((nz, ny, nx), 1.7)
    Ci = inputs.ci_random(nx, ny, nz)
    _dx, _dy, _dz = inputs.inverse_spacing(nx, ny, nz)
    dt = oracle_mod.stable_dt(1 / (nx - 1), 1 / (ny - 1), 1 / (nz - 1), 1.0, oracle_mod.maximum(Ci))
    T = oracle_mod.run(T0, Ci, 1.0, dt, _dx, _dy, _dz, 5, explicit=True)
    assert np.all(T == 1.7)


@pytest.mark.parametrize("shape,k,c", [((17, 12, 9), (1, 1, 1), 1.7), ((10, 14, 19), (3, 2, 1), 0.0)])
def test_eigenmode_decay_factor(oracle_mod, shape, k, c):
    nx, ny, nz = shape
    lam, Ci0 = 1.0, 0.5
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    xs = [np.arange(n) * d for n, d in ((nx, dx), (ny, dy), (nz, dz))]
    sx, sy, sz = (np.sin(kd * np.pi * x) for kd, x in zip(k, xs))
    mode = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    mode[~interior_mask(nx, ny, nz).reshape(nz, ny, nx)] = 0.0
    T0 = c + mode
    Ci = np.full(T0.shape, Ci0)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci0 / 6.1
    g = 1.0 - dt * lam * Ci0 * sum(4.0 / d ** 2 * np.sin(kd * np.pi * d / 2) ** 2
                                    for kd, d in zip(k, (dx, dy, dz)))
    nt = int(np.clip(round(np.log(0.05) / np.log(g)), 3, 400))
    T = oracle_mod.run(T0, Ci, lam, dt, 1 / dx, 1 / dy, 1 / dz, nt, explicit=True)
    assert np.max(np.abs(T - (c + g ** nt * mode))) <= 1e-13 * max(abs(c), 1.0)


@pytest.mark.parametrize("shape,nt", [((5, 7, 6), 7), ((8, 5, 3), 5)])
def test_dense_matrix_forward(oracle_mod, shape, nt):
    nx, ny, nz = shape
    T0, Ci, dt, (_dx, _dy, _dz) = small_problem(nx, ny, nz, seed=57 + nx, lam=LAM)
    M = dense_step_matrix(Ci, LAM, dt, _dx, _dy, _dz)
    v = T0.ravel().copy()
    for _ in range(nt):
        v = M @ v
    T = oracle_mod.run(T0, Ci, LAM, dt, _dx, _dy, _dz, nt, explicit=True)
    assert rel_linf(T.ravel(), v) <= 1e-14


def test_step_equals_run_and_writes_interior_only(oracle_mod):
    T0, Ci, dt, inv = small_problem(9, 8, 7, seed=5)
    T2 = np.full_like(T0, -1.0)
    oracle_mod.step(T2, T0, Ci, 1.0, dt, *inv, explicit=True)
    inner = interior_mask(9, 8, 7).reshape(T0.shape)
    assert np.all(T2[~inner] == -1.0)
    T2[~inner] = T0[~inner]
    assert np.array_equal(T2, oracle_mod.run(T0, Ci, 1.0, dt, *inv, 1, explicit=True))


def test_notations_agree_to_rounding(oracle_mod):
    """Fig. 1's @d2_xi form and the explicit form on the workload's fields: every
    step's results differ by rounding only (each node's difference is a few units
    in the last place of the field's scale per step), and they do differ."""
    nx, ny, nz = 24, 20, 18
    T0 = inputs.t0_gaussian(nx, ny, nz)
    Ci = inputs.ci_random(nx, ny, nz)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / Ci.max() / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    differ = False
    for nt in (1, 10, 40):
        a = oracle_mod.run(T0, Ci, 1.0, dt, *inv, nt)
        b = oracle_mod.run(T0, Ci, 1.0, dt, *inv, nt, explicit=True)
        assert np.max(np.abs(a - b)) <= nt * 8 * np.finfo(float).eps * np.max(np.abs(a))
        differ = differ or not np.array_equal(a, b)
    assert differ
