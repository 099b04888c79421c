"""Pins of the 2-D oracle (the 2-D form of Fig. 1's step: the z term dropped).

Each check is an independent formulation: the constant field (every second
difference vanishes), the discrete Dirichlet sine eigenmode's closed-form decay,
the dense step matrix built from Kronecker products, and the pinned 3-D oracle on
a grid three planes deep with a zero z-factor (its middle plane is the 2-D
problem).  A dropped term, a swapped axis or a wrong spacing fails one of them.
CPU only.
"""
import numpy as np
import pytest

from paper_2211_15634_gb300 import inputs


def second_difference_1d(n):
    D = np.zeros((n, n))
    for i in range(1, n - 1):
        D[i, i - 1], D[i, i], D[i, i + 1] = 1.0, -2.0, 1.0
    return D


def interior2d(nx, ny):
    m = np.zeros((ny, nx), dtype=bool)
    m[1:-1, 1:-1] = True
    return m


def problem2d(nx, ny, seed, lam=1.0):
    Ci = inputs.ci_random(nx, ny, 1, seed=seed)[0]
    T0 = 1.7 + inputs.random_field((ny, nx), seed + 1, 0.0, 1.0)
    dx, dy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    dt = min(dx * dx, dy * dy) / lam / Ci.max() / 4.1
    return T0, Ci, dt, (1.0 / dx, 1.0 / dy)


LAM = 0.8


def test_constant_field_stays_bitwise(oracle_mod):
    nx, ny = 13, 9
    _, Ci, dt, inv = problem2d(nx, ny, 5)
    T0 = np.full((ny, nx), 1.7)
    for nt in (3, 4):
        assert np.all(oracle_mod.run2d(T0, Ci, LAM, dt, *inv, nt) == 1.7)


@pytest.mark.parametrize("shape,k,c", [((17, 12), (1, 1), 1.7), ((21, 14), (3, 2), 0.0),
                                       ((9, 30), (2, 5), 1.7)])
def test_eigenmode_decay_factor(oracle_mod, shape, k, c):
    """g = 1 - dt*lam*Ci*(4/dx^2 sin^2(kx*pi*dx/2) + 4/dy^2 sin^2(ky*pi*dy/2)) per step."""
    nx, ny = shape
    lam, Ci0 = 1.0, 0.5
    dx, dy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    sx = np.sin(k[0] * np.pi * np.arange(nx) * dx)
    sy = np.sin(k[1] * np.pi * np.arange(ny) * dy)
    mode = sy[:, None] * sx[None, :]
    mode[~interior2d(nx, ny)] = 0.0
    T0 = c + mode
    Ci = np.full(T0.shape, Ci0)
    dt = min(dx * dx, dy * dy) / lam / Ci0 / 4.1
    g = 1.0 - dt * lam * Ci0 * (4.0 / dx ** 2 * np.sin(k[0] * np.pi * dx / 2) ** 2 +
                                4.0 / dy ** 2 * np.sin(k[1] * np.pi * dy / 2) ** 2)
    nt = int(np.clip(round(np.log(0.05) / np.log(g)), 3, 400))
    T = oracle_mod.run2d(T0, Ci, lam, dt, 1 / dx, 1 / dy, nt)
    assert np.max(np.abs(T - (c + g ** nt * mode))) <= 1e-13 * max(abs(c), 1.0)
    measured = np.sum((T - c) * mode) / np.sum(mode * mode)
    assert abs(measured - g ** nt) <= 1e-11 * g ** nt


@pytest.mark.parametrize("shape,nt", [((5, 7), 6), ((8, 3), 5), ((3, 3), 4), ((9, 6), 7)])
def test_dense_matrix_forward(oracle_mod, shape, nt):
    nx, ny = shape
    T0, Ci, dt, (_dx, _dy) = problem2d(nx, ny, 40 + nx, lam=LAM)
    L = (_dx * _dx) * np.kron(np.eye(ny), second_difference_1d(nx)) + \
        (_dy * _dy) * np.kron(second_difference_1d(ny), np.eye(nx))
    m = interior2d(nx, ny).ravel()
    L[~m, :] = 0.0
    M = np.eye(nx * ny) + (dt * LAM * Ci.ravel() * m)[:, None] * L
    v = T0.ravel().copy()
    for _ in range(nt):
        v = M @ v
    T = oracle_mod.run2d(T0, Ci, LAM, dt, _dx, _dy, nt)
    assert np.max(np.abs(T.ravel() - v)) <= 1e-14 * np.max(np.abs(v))


@pytest.mark.parametrize("shape", [(7, 5), (12, 9), (4, 3)])
def test_matches_3d_oracle_middle_plane(oracle_mod, shape):
    """The pinned 3-D oracle on a (3, ny, nx) grid with _dz = 0: its middle plane
    takes the 2-D step (the z term is d2z*0 = 0; the planes above and below are
    boundary)."""
    nx, ny = shape
    T0, Ci, dt, (_dx, _dy) = problem2d(nx, ny, 90 + nx, lam=LAM)
    T3 = np.stack([T0 + 0.3, T0, T0 - 0.2])
    C3 = np.stack([Ci, Ci, Ci])
    out3 = oracle_mod.run(T3, C3, LAM, dt, _dx, _dy, 0.0, 5)
    out2 = oracle_mod.run2d(T0, Ci, LAM, dt, _dx, _dy, 5)
    assert np.array_equal(out3[1], out2)


def test_step_writes_interior_only(oracle_mod):
    nx, ny = 10, 7
    T0, Ci, dt, inv = problem2d(nx, ny, 3)
    T2 = np.full_like(T0, -5.0)
    oracle_mod.step2d(T2, T0, Ci, 1.0, dt, *inv)
    assert np.all(T2[~interior2d(nx, ny)] == -5.0) and np.all(T2[interior2d(nx, ny)] != -5.0)


@pytest.mark.parametrize("shape", [(17, 17), (31, 9), (8, 40)])
def test_stable_dt2d_is_just_inside_the_stability_bound(oracle_mod, shape):
    """The 2-D dt keeps the explicit scheme stable with a small margin: the
    highest-frequency Dirichlet mode (a checkerboard in the interior) decays under
    the oracle's dt.  On equal spacings it grows under 1.06 times that dt (the
    margin is small); on unequal spacings it grows under the dt the larger spacing
    would give (the smaller spacing sets dt)."""
    nx, ny = shape
    lam, Ci0 = 0.7, 0.45
    dx, dy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    Ci = np.full((ny, nx), Ci0)
    dt = oracle_mod.stable_dt2d(dx, dy, lam, oracle_mod.maximum(Ci))
    kx, ky = nx - 2, ny - 2  # highest interior frequencies
    sx = np.sin(kx * np.pi * np.arange(nx) * dx)
    sy = np.sin(ky * np.pi * np.arange(ny) * dy)
    mode = sy[:, None] * sx[None, :]
    mode[~interior2d(nx, ny)] = 0.0
    amp = np.max(np.abs(mode))
    nt = 40
    stable = oracle_mod.run2d(mode, Ci, lam, dt, 1 / dx, 1 / dy, nt)
    assert np.max(np.abs(stable)) < amp
    grow = 1.06 if nx == ny else max(dx, dy) ** 2 / min(dx, dy) ** 2
    unstable = oracle_mod.run2d(mode, Ci, lam, grow * dt, 1 / dx, 1 / dy, nt)
    assert np.max(np.abs(unstable)) > amp
