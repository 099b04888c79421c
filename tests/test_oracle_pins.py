"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses an independent
formulation (a closed form, a dense matrix built from Kronecker products,
complex-step differentiation, brute force) chosen so that a dropped term, a
wrong sign, a swapped axis or a wrong spacing fails at least one of them.
CPU only.
"""
import json
import os

import numpy as np
import pytest

from paper_2211_15634_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ---------------------------------------------------------------- dense form
def second_difference_1d(n):
    """1-D three-point second difference rows for nodes 1..n-2 (boundary rows zero)."""
    D = np.zeros((n, n))
    for i in range(1, n - 1):
        D[i, i - 1], D[i, i], D[i, i + 1] = 1.0, -2.0, 1.0
    return D


def interior_mask(nx, ny, nz):
    m = np.zeros((nz, ny, nx), dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m.ravel()


def dense_laplacian(nx, ny, nz, _dx, _dy, _dz):
    """Laplacian rows at interior nodes, zero rows on the boundary (x fastest)."""
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Lx = np.kron(Iz, np.kron(Iy, second_difference_1d(nx)))
    Ly = np.kron(Iz, np.kron(second_difference_1d(ny), Ix))
    Lz = np.kron(second_difference_1d(nz), np.kron(Iy, Ix))
    L = (_dx * _dx) * Lx + (_dy * _dy) * Ly + (_dz * _dz) * Lz
    L[~interior_mask(nx, ny, nz), :] = 0.0
    return L


def dense_step_matrix(Ci, lam, dt, _dx, _dy, _dz):
    """M = I + diag(dt*lam*Ci on interior) * L: one step of Fig. 1 as a matrix."""
    nz, ny, nx = Ci.shape
    L = dense_laplacian(nx, ny, nz, _dx, _dy, _dz)
    c = dt * lam * Ci.ravel() * interior_mask(nx, ny, nz)
    return np.eye(nx * ny * nz) + c[:, None] * L


def small_problem(nx, ny, nz, seed, lam=1.0):
    Ci = inputs.ci_random(nx, ny, nz, seed=seed)
    T0 = 1.7 + inputs.random_field((nz, ny, nx), seed + 1, 0.0, 1.0)
    _dx, _dy, _dz = inputs.inverse_spacing(nx, ny, nz)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci.max() / 6.1
    return T0, Ci, dt, (_dx, _dy, _dz)


LAM = 0.8  # a conductivity other than 1 so that a dropped lam shows


# ------------------------------------------------------------------- tests
def test_golden_constant_field_stays_bitwise(oracle_mod):
    """Fig. 1's own fields: T = 1.7 everywhere stays exactly 1.7 (every d2 is 0)."""
    g = json.load(open(os.path.join(GOLDEN, "fig1_setup.json")))
    nx, ny, nz = 11, 9, 7  # small stand-in for 512^3; the invariant does not depend on n
    T0 = np.full((nz, ny, nx), g["T_initial"])
    Ci = inputs.ci_random(nx, ny, nz)  # any Ci: the invariant holds for variable Ci too
    _dx, _dy, _dz = inputs.inverse_spacing(nx, ny, nz)
    dt = oracle_mod.stable_dt(1 / (nx - 1), 1 / (ny - 1), 1 / (nz - 1), g["lam"], oracle_mod.maximum(Ci))
    for nt in (4, 5):
        T = oracle_mod.run(T0, Ci, g["lam"], dt, _dx, _dy, _dz, nt)
        assert np.all(T == g["expected"]["T_final_all_equal"])


@pytest.mark.parametrize("shape,k,c", [
    ((17, 12, 9), (1, 1, 1), 1.7),
    ((17, 12, 9), (2, 1, 3), 0.0),
    ((10, 14, 19), (3, 2, 1), 1.7),
    ((9, 9, 9), (2, 3, 1), 0.0),
])
def test_eigenmode_decay_factor(oracle_mod, shape, k, c):
    """Discrete Dirichlet sine mode: each step multiplies it by
    g = 1 - dt*lam*Ci*sum_d 4/dd^2 sin^2(k_d*pi*dd/2)  (constant Ci)."""
    nx, ny, nz = shape
    lam, Ci0, a = 1.0, 0.5, 1.0
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    xs = [np.arange(n) * d for n, d in ((nx, dx), (ny, dy), (nz, dz))]
    sx, sy, sz = (np.sin(kd * np.pi * x) for kd, x in zip(k, xs))
    mode = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    bmask = ~interior_mask(nx, ny, nz).reshape(nz, ny, nx)
    mode[bmask] = 0.0  # sin(k*pi) is 0 exactly on the boundary
    T0 = c + a * mode
    Ci = np.full(T0.shape, Ci0)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci0 / 6.1
    g = 1.0 - dt * lam * Ci0 * sum(4.0 / d ** 2 * np.sin(kd * np.pi * d / 2) ** 2
                                    for kd, d in zip(k, (dx, dy, dz)))
    _dx, _dy, _dz = 1 / dx, 1 / dy, 1 / dz
    # enough steps to decay the mode to about 5%, so a wrong factor shows clearly
    nt = int(np.clip(round(np.log(0.05) / np.log(g)), 3, 400))
    T = oracle_mod.run(T0, Ci, lam, dt, _dx, _dy, _dz, nt)
    expect = c + a * g ** nt * mode
    # rounding noise of the initial field sits in slower modes: bound it by the initial scale
    assert np.max(np.abs(T - expect)) <= 1e-13 * max(abs(c), a)
    measured = np.sum((T - c) * mode) / np.sum(mode * mode)
    assert abs(measured - g ** nt) <= 1e-11 * g ** nt


@pytest.mark.parametrize("shape,nt", [((5, 7, 6), 7), ((4, 4, 4), 6), ((8, 5, 3), 5), ((3, 3, 3), 4)])
def test_dense_matrix_forward(oracle_mod, shape, nt):
    """Oracle run == M^nt T0 with M built from Kronecker products (anisotropic grids)."""
    nx, ny, nz = shape
    T0, Ci, dt, (_dx, _dy, _dz) = small_problem(nx, ny, nz, seed=31 + nx, lam=LAM)
    M = dense_step_matrix(Ci, LAM, dt, _dx, _dy, _dz)
    v = T0.ravel().copy()
    for _ in range(nt):
        v = M @ v
    T = oracle_mod.run(T0, Ci, LAM, dt, _dx, _dy, _dz, nt)
    assert rel_linf(T.ravel(), v) <= 1e-14


@pytest.mark.parametrize("shape", [(5, 7, 6), (8, 5, 3), (3, 4, 5)])
def test_dense_matrix_adjoint(oracle_mod, shape):
    """Tbar == M^T ybar and the Ci term == dt*lam*ybar*(L T) on interior nodes."""
    nx, ny, nz = shape
    T, Ci, dt, (_dx, _dy, _dz) = small_problem(nx, ny, nz, seed=77 + ny, lam=LAM)
    ybar = inputs.random_field(T.shape, 5)
    M = dense_step_matrix(Ci, LAM, dt, _dx, _dy, _dz)
    L = dense_laplacian(nx, ny, nz, _dx, _dy, _dz)
    Cibar = np.zeros_like(T)
    Tbar = oracle_mod.adjoint_step(ybar, T, Ci, Cibar, LAM, dt, _dx, _dy, _dz)
    assert rel_linf(Tbar.ravel(), M.T @ ybar.ravel()) <= 1e-14
    expect = dt * LAM * ybar.ravel() * (L @ T.ravel())
    assert np.max(np.abs(Cibar.ravel() - expect)) <= 1e-13 * np.max(np.abs(expect))
    # accumulation: a second call adds the same term again
    oracle_mod.adjoint_step(ybar, T, Ci, Cibar, LAM, dt, _dx, _dy, _dz)
    assert np.max(np.abs(Cibar.ravel() - 2 * expect)) <= 1e-13 * np.max(np.abs(expect))


def test_complex_step_gradient(oracle_mod):
    """dL/dCi and dL/dT0 against complex-step derivatives of the dense form."""
    nx, ny, nz, nt = 4, 5, 6, 3
    T0, Ci, dt, (_dx, _dy, _dz) = small_problem(nx, ny, nz, seed=101, lam=LAM)
    Tobs = 1.7 + inputs.random_field(T0.shape, 202, 0.0, 1.0)
    L_or, dT0, dCi = oracle_mod.gradient(T0, Ci, Tobs, LAM, dt, _dx, _dy, _dz, nt)

    def loss_dense(ci_flat, t0_flat):
        M = dense_step_matrix(ci_flat.reshape(T0.shape), LAM, dt, _dx, _dy, _dz)
        v = t0_flat
        for _ in range(nt):
            v = M @ v
        r = v - Tobs.ravel()
        return 0.5 * np.sum(r * r)

    h = 1e-30
    ci = Ci.ravel().astype(complex)
    t0 = T0.ravel().astype(complex)
    assert abs(loss_dense(ci, t0).real - L_or) <= 1e-13 * L_or
    gci = np.zeros(Ci.size)
    gt0 = np.zeros(T0.size)
    for q in range(Ci.size):
        e = np.zeros(Ci.size, dtype=complex)
        e[q] = 1j * h
        gci[q] = loss_dense(ci + e, t0).imag / h
        gt0[q] = loss_dense(ci, t0 + e).imag / h
    assert rel_linf(dCi.ravel(), gci) <= 1e-12
    assert rel_linf(dT0.ravel(), gt0) <= 1e-12
    assert np.all(dCi[~interior_mask(nx, ny, nz).reshape(T0.shape)] == 0.0)


def test_adjoint_dot_product(oracle_mod):
    """<M x, y> == <x, M^T y> with M the oracle step and M^T the oracle adjoint."""
    nx, ny, nz = 13, 11, 9
    _, Ci, dt, (_dx, _dy, _dz) = small_problem(nx, ny, nz, seed=3)
    x = inputs.random_field((nz, ny, nx), 11)
    y = inputs.random_field((nz, ny, nx), 12)
    Mx = x.copy()
    oracle_mod.step(Mx, x, Ci, 1.0, dt, _dx, _dy, _dz)
    MTy = oracle_mod.adjoint_step(y, x, Ci, np.zeros_like(x), 1.0, dt, _dx, _dy, _dz)
    lhs, rhs = float(np.dot(Mx.ravel(), y.ravel())), float(np.dot(x.ravel(), MTy.ravel()))
    assert abs(lhs - rhs) <= 1e-14 * np.linalg.norm(Mx) * np.linalg.norm(y)


def test_finite_difference_gradient_16(oracle_mod):
    """Directional derivatives of L against central differences on 16^3 (rel 1e-6)."""
    n, nt, lam = 16, 20, 1.0
    T0 = inputs.t0_gaussian(n, n, n)
    Ci_true = inputs.ci_smooth(n, n, n)
    Ci = inputs.ci_constant(n, n, n) + 0.01 * inputs.random_field((n, n, n), 8)
    _dx, _dy, _dz = inputs.inverse_spacing(n, n, n)
    dx = 1.0 / (n - 1)
    dt = dx * dx / lam / (1.5 / inputs.C0) / 6.1  # dt from the bound max Ci <= 1.5/c0
    Tobs = oracle_mod.run(T0, Ci_true, lam, dt, _dx, _dy, _dz, nt)
    L, dT0, dCi = oracle_mod.gradient(T0, Ci, Tobs, lam, dt, _dx, _dy, _dz, nt)

    def L_of(ci, t0):
        return oracle_mod.loss(oracle_mod.run(t0, ci, lam, dt, _dx, _dy, _dz, nt), Tobs)

    assert abs(L_of(Ci, T0) - L) <= 1e-14 * L
    v = inputs.random_field((n, n, n), 9)
    h = 1e-4
    fd = (L_of(Ci + h * v, T0) - L_of(Ci - h * v, T0)) / (2 * h)
    ad = float(np.dot(dCi.ravel(), v.ravel()))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    w = inputs.random_field((n, n, n), 10)
    h = 1e-3
    fd = (L_of(Ci, T0 + h * w) - L_of(Ci, T0 - h * w)) / (2 * h)
    ad = float(np.dot(dT0.ravel(), w.ravel()))
    assert abs(fd - ad) <= 1e-6 * abs(ad)


def test_maximum_brute_force(oracle_mod):
    a = inputs.random_field((7, 6, 5), 44, -3.0, 2.0)
    assert oracle_mod.maximum(a) == max(a.ravel().tolist())
    a[3, 2, 1] = 9.5
    assert oracle_mod.maximum(a) == 9.5


def test_stable_dt_paper_setup_and_max_principle(oracle_mod):
    """Fig. 1 dt with Ci = 1/c0 at 512^3; the resulting step never exceeds the data's range."""
    g = json.load(open(os.path.join(GOLDEN, "fig1_setup.json")))
    dx = g["lx"] / (g["nx"] - 1)
    dt = oracle_mod.stable_dt(dx, dx, dx, g["lam"], 1.0 / g["c0"])
    # with Ci = 1/c0 the update weight on each neighbour is dt*lam*Ci/dx^2 = 1/6.1
    assert abs(dt * g["lam"] * (1.0 / g["c0"]) / (dx * dx) - 1.0 / 6.1) <= 1e-15
    # anisotropic: the smallest spacing wins, and the step is a convex combination
    nx, ny, nz = 11, 21, 6
    Ci = inputs.ci_random(nx, ny, nz)
    sp = inputs.spacing(nx, ny, nz)
    dt = oracle_mod.stable_dt(*sp, 1.0, oracle_mod.maximum(Ci))
    assert dt == min(d * d for d in sp) / 1.0 / Ci.max() / 6.1
    T = inputs.random_field((nz, ny, nx), 4, 0.0, 1.0)
    T2 = T.copy()
    oracle_mod.step(T2, T, Ci, 1.0, dt, *[1 / d for d in sp])
    assert T2.min() >= T.min() - 1e-15 and T2.max() <= T.max() + 1e-15


def test_step_writes_interior_only(oracle_mod):
    nx, ny, nz = 6, 5, 4
    T, Ci, dt, inv = small_problem(nx, ny, nz, seed=9)
    T2 = np.full_like(T, np.nan)
    oracle_mod.step(T2, T, Ci, 1.0, dt, *inv)
    inner = interior_mask(nx, ny, nz).reshape(T.shape)
    assert np.all(np.isnan(T2[~inner])) and np.all(np.isfinite(T2[inner]))


@pytest.mark.parametrize("nt", [0, 1, 2, 5])
def test_run_equals_repeated_steps(oracle_mod, nt):
    """run = T2 = copy(T) followed by nt step-and-swap rounds (Fig. 1 time loop)."""
    nx, ny, nz = 7, 6, 5
    T0, Ci, dt, inv = small_problem(nx, ny, nz, seed=19)
    cur, nxt = T0.copy(), T0.copy()
    for _ in range(nt):
        oracle_mod.step(nxt, cur, Ci, 1.0, dt, *inv)
        cur, nxt = nxt, cur
    assert np.array_equal(oracle_mod.run(T0, Ci, 1.0, dt, *inv, nt), cur)


def test_threads_do_not_change_results(oracle_mod):
    """The OpenMP split over z is a pure partition: results are bit-identical."""
    nx, ny, nz = 20, 18, 16
    T0, Ci, dt, inv = small_problem(nx, ny, nz, seed=23)
    oracle_mod.set_threads(1)
    a = oracle_mod.run(T0, Ci, 1.0, dt, *inv, 5)
    oracle_mod.set_threads(max(2, oracle_mod.max_threads()))
    b = oracle_mod.run(T0, Ci, 1.0, dt, *inv, 5)
    oracle_mod.set_threads(1)
    assert np.array_equal(a, b)
