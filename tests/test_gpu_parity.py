"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
* FP64: relative L-inf <= 1e-12 after nt steps (measured against max|T_ref|).
* FP32 (deviation storage): |D_gpu - D_ref| <= nt * 13 * 2^-24 * max|D0|, the
  worst-case bound of one FP32 rounding of D + delta plus about six roundings
  inside delta (|delta| <= 2 max|D| for a stable dt) per step, with errors
  carried forward without growth by the contractive step.  The reference is
  the FP64 oracle run on the FP32-rounded Ci and D0, so the bound covers the
  arithmetic only; storage rounding is reported separately by the benchmark.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import light_cone_reference, problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

U32 = 2.0 ** -24
FP64_TOL = 1e-12


def f32_tol(nt, D0):
    return nt * 13 * U32 * float(np.max(np.abs(D0)))


def gpu_run(T0, Ci, lam, dt, inv, nt, dtype=torch.float64, **kw):
    T = to_dev(T0, dtype)
    T2 = torch.empty_like(T)
    C = to_dev(Ci, dtype)
    res = api.run(T, T2, C, lam, dt, inv, nt, **kw)
    return to_host(res)


# odd nx -> plain column kernel; nx*8 % 16 == 0 -> TMA z-march (64 x 8 tiles in FP64,
# 128 x 8 in FP32): several tiles in x and y with ragged tails, and short z ranges
SHAPES = [(3, 3, 3), (4, 3, 5), (5, 6, 7), (37, 29, 23), (66, 19, 20), (130, 67, 33), (257, 9, 12),
          (132, 21, 17), (256, 35, 19), (68, 70, 40), (200, 3, 4)]
F32_SHAPES = [(5, 6, 7), (37, 29, 23), (130, 67, 33), (132, 21, 17), (256, 35, 19), (4, 9, 5)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nt", [1, 2, 9])
def test_fp64_run_matches_oracle(shape, nt):
    nx, ny, nz = shape
    T0, Ci, lam, dt, inv = problem(nx, ny, nz, gaussian=False)
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    got = gpu_run(T0, Ci, lam, dt, inv, nt)
    assert rel_linf(got, ref) <= FP64_TOL


@pytest.mark.parametrize("shape", [(37, 29, 23), (130, 67, 33)])
def test_fp64_native_kernel_matches_oracle(shape):
    nx, ny, nz = shape
    T0, Ci, lam, dt, inv = problem(nx, ny, nz)
    ref = oracle.run(T0, Ci, lam, dt, *inv, 20)
    got = gpu_run(T0, Ci, lam, dt, inv, 20, native_f64=True)
    assert rel_linf(got, ref) <= FP64_TOL


def test_fp64_step_leaves_boundary_untouched():
    nx, ny, nz = 21, 18, 13
    T0, Ci, lam, dt, inv = problem(nx, ny, nz)
    T = to_dev(T0)
    T2 = torch.full_like(T, float("nan"))
    api.step(T2, T, to_dev(Ci), lam, dt, inv)
    out = to_host(T2)
    inner = np.zeros(T0.shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.all(np.isnan(out[~inner])) and np.all(np.isfinite(out[inner]))
    ref = T0.copy()
    oracle.step(ref, T0, Ci, lam, dt, *inv)
    assert rel_linf(out[inner], ref[inner]) <= 1e-15


def test_constant_field_stays_bitwise_fp64_and_fp32():
    nx, ny, nz = 67, 35, 19
    _, Ci, lam, dt, inv = problem(nx, ny, nz)
    T0 = np.full((nz, ny, nx), 1.7)
    assert np.all(gpu_run(T0, Ci, lam, dt, inv, 7) == 1.7)
    D0 = np.zeros((nz, ny, nx))  # deviation of the constant field
    assert np.all(gpu_run(D0, Ci, lam, dt, inv, 7, dtype=torch.float32) == 0.0)


@pytest.mark.parametrize("shape,k", [((33, 20, 17), (1, 2, 1)), ((64, 64, 64), (2, 1, 3))])
def test_eigenmode_decay_on_gpu(shape, k):
    nx, ny, nz = shape
    lam, Ci0, nt = 1.0, 0.5, 40
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    s = [np.sin(kd * np.pi * np.arange(n) * d) for kd, n, d in zip(k, (nx, ny, nz), (dx, dy, dz))]
    mode = s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]
    mode[[0, -1], :, :] = 0.0
    mode[:, [0, -1], :] = 0.0
    mode[:, :, [0, -1]] = 0.0
    T0 = 1.7 + mode
    Ci = np.full(T0.shape, Ci0)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci0 / 6.1
    g = 1.0 - dt * lam * Ci0 * sum(4.0 / d ** 2 * np.sin(kd * np.pi * d / 2) ** 2
                                    for kd, d in zip(k, (dx, dy, dz)))
    got = gpu_run(T0, Ci, lam, dt, (1 / dx, 1 / dy, 1 / dz), nt)
    assert np.max(np.abs(got - (1.7 + g ** nt * mode))) <= 1e-13 * 2.7


def test_run_graph_equals_plain_run_bitwise():
    nx, ny, nz = 70, 41, 29
    T0, Ci, lam, dt, inv = problem(nx, ny, nz)
    a = gpu_run(T0, Ci, lam, dt, inv, 11)
    b = gpu_run(T0, Ci, lam, dt, inv, 11, graph=True)
    c = gpu_run(T0, Ci, lam, dt, inv, 11, graph=True)  # cached graph replay
    assert np.array_equal(a, b) and np.array_equal(a, c)
    api.clear_graph_cache()


def test_run_nt0_returns_input():
    T0, Ci, lam, dt, inv = problem(9, 8, 7)
    assert np.array_equal(gpu_run(T0, Ci, lam, dt, inv, 0), T0)


# ------------------------------------------------------- pre-scaled coefficient
def iso_problem(nx, ny, nz, gaussian=False):
    """Workload fields on a grid with one spacing d in every direction."""
    T0, Ci, lam, _, _ = problem(nx, ny, nz, gaussian=gaussian)
    d = 1.0 / (max(nx, ny, nz) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, (1.0 / d,) * 3


def prescaled_run(T0, Ci, lam, dt, inv, nt, **kw):
    T = to_dev(T0)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    return to_host(api.run(T, torch.empty_like(T), Cs, lam, dt, inv, nt, ci_scaled=True, **kw))


@pytest.mark.parametrize("shape", [(3, 3, 3), (5, 6, 7), (37, 29, 23), (66, 19, 20), (130, 67, 33),
                                   (256, 35, 19), (68, 70, 40)])
@pytest.mark.parametrize("nt", [1, 9])
def test_fp64_prescaled_ci_matches_oracle(shape, nt):
    """Cs = dt*lam*_d^2*Ci once, then T2 = T + Cs*(sum of neighbours - 6T):
    the same step on a grid with equal spacings."""
    T0, Ci, lam, dt, inv = iso_problem(*shape)
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    assert rel_linf(prescaled_run(T0, Ci, lam, dt, inv, nt), ref) <= FP64_TOL
    assert api.device_error() == 0


@pytest.mark.parametrize("shape", [(37, 29, 23), (130, 67, 33)])
def test_fp64_matches_both_notations(shape):
    """The paper's Results run Fig. 1's solver and an explicit-notation one (second
    differences written A[i+1] - 2*A[i] + A[i-1]): one operator, different roundings.
    The FP64 step forms the neighbour sum exactly, so it is within 1e-12 of the
    oracle in either notation (pre-scaled and on Ci as given)."""
    nt = 9
    T0, Ci, lam, dt, inv = iso_problem(*shape)
    got_s = prescaled_run(T0, Ci, lam, dt, inv, nt)
    T = to_dev(T0)
    got_c = to_host(api.run(T, torch.empty_like(T), to_dev(Ci), lam, dt, inv, nt))
    for explicit in (False, True):
        ref = oracle.run(T0, Ci, lam, dt, *inv, nt, explicit=explicit)
        assert rel_linf(got_s, ref) <= FP64_TOL
        assert rel_linf(got_c, ref) <= FP64_TOL
    assert api.device_error() == 0


def test_fp64_prescaled_general_path_and_graph():
    """Signs, zeros and binade changes (fixed-point path) with the pre-scaled
    coefficient, run plainly and as a CUDA graph (bitwise equal)."""
    nx, ny, nz, nt = 64, 31, 17, 6
    _, Ci, lam, dt, inv = iso_problem(nx, ny, nz)
    T0 = inputs.random_field((nz, ny, nx), 78, -1.0, 1.0)
    T0[::3, :, ::5] = 0.0
    T0[1::4, ::2, :] *= 1e-9
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    a = prescaled_run(T0, Ci, lam, dt, inv, nt)
    b = prescaled_run(T0, Ci, lam, dt, inv, nt, graph=True)
    assert rel_linf(a, ref) <= FP64_TOL and np.array_equal(a, b)
    api.clear_graph_cache()


def test_fp64_prescaled_step_kernel_and_in_place_scale():
    nx, ny, nz = 64, 20, 12
    T0, Ci, lam, dt, inv = iso_problem(nx, ny, nz, gaussian=True)
    T, C = to_dev(T0), to_dev(Ci)
    T2 = torch.empty_like(T)
    api.copy_boundary(T2, T)
    assert api.step_kernel_name(T2, T, C, lam, dt, inv, ci_scaled=True) == "k_zmarch<F64_SCALED4>"
    api.scale_ci(C, lam, dt, inv, out=C)  # in place
    api.step(T2, T, C, lam, dt, inv, ci_scaled=True)
    ref = T0.copy()
    oracle.step(ref, T0, Ci, lam, dt, *inv)
    assert rel_linf(to_host(T2), ref) <= 1e-15
    with pytest.raises(Exception, match="equal spacings"):
        api.step(T2, T, C, lam, dt, (inv[0], inv[1], inv[2] * 2), ci_scaled=True)


# --------------------------------------------------------------------- FP32
@pytest.mark.parametrize("kchunk", ["1", "3", "7"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_short_z_chunks(launch_override, kchunk, dtype):
    """Many z-chunks per column (pipeline prologue/epilogue at every chunk edge)."""
    launch_override(kchunk=kchunk)
    nx, ny, nz, nt = 136, 27, 22, 5
    T0, Ci, lam, dt, inv = problem(nx, ny, nz)
    if dtype == torch.float64:
        ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
        assert rel_linf(gpu_run(T0, Ci, lam, dt, inv, nt), ref) <= FP64_TOL
    else:
        D0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
        C32 = Ci.astype(np.float32).astype(np.float64)
        ref = oracle.run(D0, C32, lam, dt, *inv, nt)
        got = gpu_run(D0, C32, lam, dt, inv, nt, dtype=torch.float32)
        assert np.max(np.abs(got - ref)) <= f32_tol(nt, D0)
    assert api.device_error() == 0


def test_emulated_fp64_general_path():
    """Fields that cross zero and binades at every node (signs, zeros, tiny
    values) exercise the fixed-point path of the one-DFMA arithmetic."""
    nx, ny, nz, nt = 66, 31, 17, 6
    _, Ci, lam, dt, inv = problem(nx, ny, nz)
    T0 = inputs.random_field((nz, ny, nx), 77, -1.0, 1.0)
    T0[::3, :, ::5] = 0.0
    T0[1::4, ::2, :] *= 1e-9
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    for flags in ({}, {"native_f64": True}):
        assert rel_linf(gpu_run(T0, Ci, lam, dt, inv, nt, **flags), ref) <= FP64_TOL


@pytest.mark.parametrize("shape", F32_SHAPES)
@pytest.mark.parametrize("comp", [False, True])
def test_fp32_run_matches_oracle(shape, comp):
    nx, ny, nz = shape
    nt = 20
    T0, Ci, lam, dt, inv = problem(nx, ny, nz)
    D0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
    Ci32 = Ci.astype(np.float32).astype(np.float64)
    ref = oracle.run(D0, Ci32, lam, dt, *inv, nt)
    D = to_dev(D0, torch.float32)
    D2 = torch.empty_like(D)
    C = to_dev(Ci32, torch.float32)
    cbuf = api.compensation_fields(D) if comp else None
    res = api.run(D, D2, C, lam, dt, inv, nt, comp=cbuf)
    got = to_host(api.from_deviation_pair(res, cbuf[nt % 2], 0.0) if comp else res)
    assert np.max(np.abs(got - ref)) <= f32_tol(nt, D0)


def test_deviation_roundtrip():
    T0, *_ = problem(31, 17, 9)
    T = to_dev(T0)
    D = api.to_deviation(T, 1.7)
    assert np.array_equal(to_host(D), (T0 - 1.7).astype(np.float32).astype(np.float64))
    back = to_host(api.from_deviation(D, 1.7))
    assert np.array_equal(back, (T0 - 1.7).astype(np.float32).astype(np.float64) + 1.7)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("shape", [(3, 3, 3), (5, 7, 6), (37, 29, 23), (66, 19, 20), (4, 5, 6),
                                   (68, 21, 19), (132, 11, 9), (256, 9, 17), (128, 16, 3)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_adjoint_step_matches_oracle(shape, dtype):
    nx, ny, nz = shape
    T, Ci, lam, dt, inv = problem(nx, ny, nz, gaussian=False)
    ybar = inputs.random_field(T.shape, 5)
    cib0 = inputs.random_field(T.shape, 6)
    if dtype == torch.float32:
        T, Ci, ybar, cib0 = (a.astype(np.float32).astype(np.float64) for a in (T, Ci, ybar, cib0))
    cib_ref = cib0.copy()
    tbar_ref = oracle.adjoint_step(ybar, T, Ci, cib_ref, lam, dt, *inv)
    Tbar = torch.empty(T.shape, dtype=dtype, device="cuda")
    Cib = to_dev(cib0, dtype)
    api.adjoint(Tbar, Cib, to_dev(ybar, dtype), to_dev(T, dtype), to_dev(Ci, dtype), lam, dt, inv)
    tol = 1e-14 if dtype == torch.float64 else 2e-6
    assert rel_linf(to_host(Tbar), tbar_ref) <= tol
    assert np.max(np.abs(to_host(Cib) - cib_ref)) <= tol * np.max(np.abs(cib_ref))


def test_gpu_adjoint_dot_product():
    nx, ny, nz = 45, 33, 27
    _, Ci, lam, dt, inv = problem(nx, ny, nz)
    x = inputs.random_field((nz, ny, nx), 11)
    y = inputs.random_field((nz, ny, nx), 12)
    xd, yd, Cd = to_dev(x), to_dev(y), to_dev(Ci)
    Mx = xd.clone()
    api.step(Mx, xd, Cd, lam, dt, inv)
    MTy = torch.empty_like(yd)
    api.adjoint(MTy, torch.zeros_like(yd), yd, xd, Cd, lam, dt, inv)
    lhs = float(api.dot(Mx, yd))
    rhs = float(api.dot(xd, MTy))
    assert abs(lhs - rhs) <= 1e-14 * float(torch.linalg.norm(Mx) * torch.linalg.norm(yd))


# --------------------------------------------------------------- reductions
@pytest.mark.parametrize("n", [1, 7, 1000, 1234567])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_reductions(n, dtype):
    a = inputs.random_field((n,), 3, -2.0, 1.0)
    b = inputs.random_field((n,), 4, -1.0, 3.0)
    if dtype == torch.float32:
        a, b = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    A, B = to_dev(a, dtype), to_dev(b, dtype)
    assert api.maximum(A) == a.max()
    assert float(api.maximum_async(A)) == a.max()
    assert abs(float(api.dot(A, B)) - float(np.dot(a, b))) <= 1e-13 * float(np.dot(np.abs(a), np.abs(b)))
    R = torch.empty_like(A)
    L = float(api.half_sq_dist(A, B, residual=R))
    assert abs(L - 0.5 * float(np.sum((a - b) ** 2))) <= 1e-13 * L
    exp_r = (a - b) if dtype == torch.float64 else (a - b).astype(np.float32).astype(np.float64)
    assert np.array_equal(to_host(R), exp_r)
    # a fixed partition and order: repeated sums are bitwise equal
    assert float(api.dot(A, B)) == float(api.dot(A, B))


def test_stable_dt_matches_oracle():
    nx, ny, nz = 40, 33, 21
    Ci = inputs.ci_random(nx, ny, nz)
    dt = api.stable_dt(to_dev(Ci), 1.0)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    assert dt == oracle.stable_dt(dx, dy, dz, 1.0, oracle.maximum(Ci))


def test_copy_boundary():
    T0, *_ = problem(19, 14, 11, gaussian=False)
    T = to_dev(T0)
    T2 = torch.full_like(T, -5.0)
    api.copy_boundary(T2, T)
    out = to_host(T2)
    inner = np.zeros(T0.shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.array_equal(out[~inner], T0[~inner]) and np.all(out[inner] == -5.0)


# -------------------------------------------------------------------- batch
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_matches_single_runs(dtype):
    sizes = [3, 5, 17, 32, 40, 33, 64]
    nt = 7
    probs, refs = [], []
    for q, n in enumerate(sizes):
        T0, Ci, lam, dt, inv = problem(n, n, n, seed=1000 + q)
        if dtype == torch.float32:
            T0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
            Ci = Ci.astype(np.float32).astype(np.float64)
        refs.append((oracle.run(T0, Ci, lam, dt, *inv, nt), T0))
        T = to_dev(T0, dtype)
        probs.append(dict(T=T, T2=T.clone(), Ci=to_dev(Ci, dtype), lam=lam, dt=dt, inv_spacing=inv))
    b = api.Batch(probs)
    b.run(nt, graph=True)
    for q, (ref, T0) in enumerate(refs):
        got = to_host(b.result(q, nt))
        if dtype == torch.float64:
            assert rel_linf(got, ref) <= FP64_TOL
        else:
            assert np.max(np.abs(got - ref)) <= f32_tol(nt, T0) + 1e-30
    api.clear_graph_cache()


def test_tuned_batch_matches_oracle(tmp_path, monkeypatch):
    """Autotuned per-size-class tiles (row-packed and fixed shapes mixed in one
    table) give the same results as the oracle; the tuner caches its choice."""
    import json
    from paper_2211_15634_gb300 import tuner
    monkeypatch.setenv("PS_TUNER_CACHE", str(tmp_path / "tuner.json"))
    sizes = [34, 47, 50, 79, 90, 131, 150]
    nt = 4
    probs, refs = [], []
    for q, n in enumerate(sizes):
        T0, Ci, lam, dt, inv = problem(n, n, n, seed=2000 + q)
        refs.append(oracle.run(T0, Ci, lam, dt, *inv, nt))
        T = to_dev(T0)
        probs.append(dict(T=T, T2=T.clone(), Ci=to_dev(Ci), lam=lam, dt=dt, inv_spacing=inv))
    best = tuner.tune(probs, reps=2)
    cache = json.load(open(tmp_path / "tuner.json"))
    assert len(cache) == len(best) and all(tuple(v) in tuner.CANDIDATES for v in cache.values())
    # reset the states (tuning stepped them) and run the tuned table
    for p, n, q in zip(probs, sizes, range(len(sizes))):
        T0, *_ = problem(n, n, n, seed=2000 + q)
        p["T"].copy_(to_dev(T0))
        p["T2"].copy_(p["T"])
    b = tuner.tuned_batch(probs)
    b.run(nt, graph=False)
    for q, ref in enumerate(refs):
        assert rel_linf(to_host(b.result(q, nt)), ref) <= FP64_TOL


# -------------------------------------------------------- full-size checks
@pytest.mark.slow
def test_fp64_512_light_cone_samples():
    """The benchmark's workload (512^3, Gaussian T0, random Ci, nt=100) in the
    launch configuration it times, checked at sampled nodes against the oracle
    on each node's dependency cone."""
    n, nt = 512, 100
    T0, Ci, lam, dt, inv = problem(n, n, n)
    got = gpu_run(T0, Ci, lam, dt, inv, nt, graph=True)
    pts = [(256, 256, 256), (1, 1, 1), (510, 300, 7), (255, 3, 509), (120, 400, 256), (0, 17, 30)]
    oracle.set_threads(max(1, oracle.max_threads()))
    ref = light_cone_reference(oracle, T0, Ci, lam, dt, inv, nt, pts)
    oracle.set_threads(1)
    vals = np.array([got[k, j, i] for (i, j, k) in pts])
    assert np.max(np.abs(vals - ref)) <= FP64_TOL * np.max(np.abs(T0))
    # the step is a convex combination: the field stays within the initial range
    assert got.min() >= T0.min() - 1e-12 and got.max() <= T0.max() + 1e-12
    api.clear_graph_cache()


@pytest.mark.slow
def test_fp64_512_one_step_samples():
    """One step at 512^3: sampled nodes against the oracle's step on each
    node's 3x3x3 neighbourhood."""
    n = 512
    T0, Ci, lam, dt, inv = problem(n, n, n)
    T = to_dev(T0)
    T2 = T.clone()
    api.step(T2, T, to_dev(Ci), lam, dt, inv)
    got = to_host(T2)
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(1, n - 1, 3)) for _ in range(2000)]
    ref = light_cone_reference(oracle, T0, Ci, lam, dt, inv, 1, pts)
    vals = np.array([got[k, j, i] for (i, j, k) in pts])
    assert np.max(np.abs(vals - ref)) <= 1e-15 * np.max(np.abs(T0))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_state_block_copies_boundary_into_every_grid(dtype):
    """One launch writes T's six faces into each of several padded grids and
    leaves their interiors alone; every grid starts on a 16-byte boundary."""
    nx, ny, nz = 7, 5, 3  # n = 105: odd, so the grids need a padded stride
    T = to_dev(inputs.random_field((nz, ny, nx), 31), dtype)
    grids = api.state_block(T, 5)
    for g in grids:
        g[1:-1, 1:-1, 1:-1] = -1.0
    grids2 = api.state_block(T, 5)
    for g in grids2:
        assert g.data_ptr() % 16 == 0
    inner = np.zeros((nz, ny, nx), dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    Th = to_host(T)
    for g in grids:
        gh = to_host(g)
        assert np.array_equal(gh[~inner], Th[~inner]) and np.all(gh[inner] == -1.0)


@pytest.mark.parametrize("every", [1, 4])
def test_run_states_graph_equals_launches(every):
    """The state-keeping loop replayed from the graph cache: every grid bit for bit the
    loop's launched one by one; the second call replays the captured graph."""
    nx, ny, nz = 68, 21, 13
    nt = 9
    T0h, Ci, lam, dt, inv = iso_problem(nx, ny, nz)
    T0 = to_dev(T0h)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    count = nt // every + (2 if every > 1 else 0)
    plain = api.StateBlock(T0, count, boundary=False)
    f0 = api.run_states(T0, plain, every, Cs, lam, dt, inv, nt, ci_scaled=True)
    api.clear_graph_cache()
    block = api.StateBlock(T0, count, boundary=False)
    for call in range(2):
        block.flat.fill_(float("nan"))
        f = api.run_states(T0, block, every, Cs, lam, dt, inv, nt, ci_scaled=True, graph=True)
        assert api.graph_cache_size() == 1, call
        for t in range(every, nt + 1, every):
            assert torch.equal(block.grids[t // every - 1], plain.grids[t // every - 1]), (call, t)
        assert torch.equal(f, f0)
    api.clear_graph_cache()
    assert api.device_error() == 0


RUN_STATES_FORMS = {  # name: (shape nx, ny, nz; dtype; pre-scaled?)
    "f64_scaled4": ((68, 21, 13), torch.float64, True),
    "f64_scaled2": ((66, 19, 13), torch.float64, True),
    "f64_as_given": ((68, 21, 13), torch.float64, False),
    "f32": ((68, 19, 13), torch.float32, False),
    "f64_column": ((67, 21, 13), torch.float64, True),  # odd nx: the plain column kernel
}


@pytest.mark.parametrize("every", [1, 4])
@pytest.mark.parametrize("form", list(RUN_STATES_FORMS))
def test_run_states_sets_the_boundary_of_unprepared_grids(form, every):
    """State grids handed to run_states with NaN everywhere: every grid the call writes
    ends, boundary included, bit for bit equal to the step loop's state (the z-march
    steps store the x and y faces, the call copies the z faces; the column kernel's
    grids get the whole boundary copied)."""
    (nx, ny, nz), dtype, scaled = RUN_STATES_FORMS[form]
    nt = 9
    T0h, Ci, lam, dt, inv = iso_problem(nx, ny, nz)
    T0 = to_dev(T0h, dtype)
    C = to_dev(Ci, dtype)
    if scaled:
        C = api.scale_ci(C, lam, dt, inv)
    block = api.StateBlock(T0, nt // every + (2 if every > 1 else 0), boundary=False)
    block.flat.fill_(float("nan"))
    final = api.run_states(T0, block, every, C, lam, dt, inv, nt, ci_scaled=scaled)
    a, b = T0.clone(), T0.clone()
    cur = a
    for t in range(1, nt + 1):
        dst = b if cur is a else a
        api.step(dst, cur, C, lam, dt, inv, ci_scaled=scaled)
        cur = dst
        if t % every == 0:
            assert torch.equal(block.grids[t // every - 1], cur), t
    assert torch.equal(final, cur)
    assert api.device_error() == 0


@pytest.mark.parametrize("nt,every", [(0, 1), (1, 1), (7, 1), (7, 3), (9, 3), (5, 8), (12, 5)])
def test_run_states_keeps_the_states_of_a_step_loop(nt, every):
    """The library's state-keeping time loop: slot t/every - 1 holds the state after
    step t (every dividing t), the returned grid holds T(nt), bit for bit the states
    of single steps; T0 is not modified."""
    nx, ny, nz = 34, 21, 17
    T0h, Ci, lam, dt, inv = problem(nx, ny, nz)
    T0 = to_dev(T0h)
    C = to_dev(Ci)
    block = api.StateBlock(T0, nt // every + (2 if every > 1 and nt > 0 else 0))
    final = api.run_states(T0, block, every, C, lam, dt, inv, nt)
    a, b = T0.clone(), T0.clone()
    api.copy_boundary(b, a)
    cur = a
    for t in range(1, nt + 1):
        dst = b if cur is a else a
        api.step(dst, cur, C, lam, dt, inv)
        cur = dst
        if t % every == 0:
            assert torch.equal(block.grids[t // every - 1], cur), t
    assert torch.equal(final, cur)
    assert np.array_equal(to_host(T0), T0h)
