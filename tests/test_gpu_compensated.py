"""The compensated FP32 step (two-float state D + E, ps_diffusion3d_step_comp_f32)
against the FP64 oracle, separately for the two sources of FP32 error:

* arithmetic error: the oracle is run on exactly the state the GPU starts from and on
  the FP32-rounded Ci, so only the step's own roundings are measured;
* storage error: the oracle is run on the FP64 T0 (Ci still the FP32 one the GPU
  reads), so rounding T0 to the stored state counts as well.

In the regime where the compensation matters - steps whose update is far below an
ulp of D (a small dt) - it must beat the plain FP32 step by orders of magnitude, and
with the workload's dt it must still be more accurate.  Also: the staged kernel
equals the plain column kernel bit for bit (the same explicitly rounded
arithmetic), graph and stream runs agree, and the pair conversions round-trip."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, to_dev, to_host
from paper_2211_15634_gb300 import api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def fp32_runs(T0, Ci, lam, dt, inv, nt, pair_start):
    """(plain result, compensated result) as FP64 absolute temperatures; the
    compensated run starts from the two-float deviation of T0 when pair_start."""
    T = to_dev(T0)
    C = api.to_f32(to_dev(Ci))
    D = api.to_deviation(T, 1.7)
    plain = to_host(api.from_deviation(api.run(D.clone(), torch.empty_like(D), C, lam, dt, inv, nt), 1.7))
    if pair_start:
        Dc, E0 = api.to_deviation_pair(T, 1.7)
    else:
        Dc, E0 = D.clone(), None
    comp = api.compensation_fields(Dc, E0)
    res = api.run(Dc, torch.empty_like(Dc), C, lam, dt, inv, nt, comp=comp)
    got = to_host(api.from_deviation_pair(res, comp[nt % 2], 1.7))
    return plain, got


def f32_inputs(T0, Ci):
    D0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
    return D0, Ci.astype(np.float32).astype(np.float64)


def err(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("shape", [(68, 40, 36), (132, 21, 17)])
def test_small_updates_arithmetic_error(shape):
    """dt a thousandth of the stable step, 1000 steps: each update is far below half
    an ulp of D, so the plain step loses most of it while the compensated step keeps it."""
    T0, Ci, lam, dt, inv = problem(*shape)
    dt *= 1e-3
    nt = 1000
    D0, C32 = f32_inputs(T0, Ci)
    ref = oracle.run(D0, C32, lam, dt, *inv, nt) + 1.7
    plain, comp = fp32_runs(T0, Ci, lam, dt, inv, nt, pair_start=False)
    e_plain, e_comp = err(plain, ref), err(comp, ref)
    assert e_comp < e_plain / 100, (e_comp, e_plain)
    assert e_comp < 1e-9


@pytest.mark.parametrize("shape", [(68, 40, 36), (132, 21, 17)])
def test_workload_dt_arithmetic_error(shape):
    """With the workload's stable dt the compensated step is still the more accurate."""
    T0, Ci, lam, dt, inv = problem(*shape)
    nt = 100
    D0, C32 = f32_inputs(T0, Ci)
    ref = oracle.run(D0, C32, lam, dt, *inv, nt) + 1.7
    plain, comp = fp32_runs(T0, Ci, lam, dt, inv, nt, pair_start=False)
    assert err(comp, ref) < 0.5 * err(plain, ref), (err(comp, ref), err(plain, ref))


def test_storage_error_with_a_two_float_start():
    """Starting from the two-float deviation of T0 removes T0's FP32 rounding: against
    the oracle on the FP64 T0 the compensated run's error is far below the plain one's."""
    T0, Ci, lam, dt, inv = problem(68, 40, 36)
    dt *= 1e-3
    nt = 200
    C32 = Ci.astype(np.float32).astype(np.float64)
    ref = oracle.run(T0, C32, lam, dt, *inv, nt)
    plain, comp = fp32_runs(T0, Ci, lam, dt, inv, nt, pair_start=True)
    assert err(comp, ref) < err(plain, ref) / 100
    assert err(comp, ref) < 1e-10


@pytest.mark.parametrize("shape", [(132, 21, 17), (64, 9, 7), (260, 37, 11)])
def test_staged_kernel_equals_plain_kernel_bitwise(launch_override, shape):
    T0, Ci, lam, dt, inv = problem(*shape, gaussian=False)
    T = to_dev(T0)
    C = api.to_f32(to_dev(Ci))
    outs = []
    for plain in (0, 1):
        launch_override(step_plain=plain)
        D, E0 = api.to_deviation_pair(T, 1.7)
        comp = api.compensation_fields(D, E0)
        res = api.run(D, torch.empty_like(D), C, lam, dt, inv, 7, comp=comp)
        outs.append((to_host(res), to_host(comp[1])))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert api.device_error() == 0


def test_graph_equals_stream_and_single_steps():
    """run(comp=..., graph=True) = the plain loop = step_compensated called nt times."""
    T0, Ci, lam, dt, inv = problem(136, 27, 22, gaussian=False)
    T = to_dev(T0)
    C = api.to_f32(to_dev(Ci))
    nt = 5
    outs = []
    for graph in (False, True):
        D, E0 = api.to_deviation_pair(T, 1.7)
        comp = api.compensation_fields(D, E0)
        res = api.run(D, torch.empty_like(D), C, lam, dt, inv, nt, comp=comp, graph=graph)
        outs.append((to_host(res), to_host(comp[nt % 2])))
    D, E = api.to_deviation_pair(T, 1.7)
    D2, E2 = D.clone(), E.clone()
    for _ in range(nt):
        api.step_compensated(D2, D, E2, E, C, lam, dt, inv)
        D, D2, E, E2 = D2, D, E2, E
    for a in outs:
        assert np.array_equal(a[0], to_host(D)) and np.array_equal(a[1], to_host(E))
    api.clear_graph_cache()


def test_deviation_pair_round_trip():
    T0, *_ = problem(31, 17, 9, gaussian=False)
    D, E = api.to_deviation_pair(to_dev(T0), 1.7)
    d = (T0 - 1.7).astype(np.float32)
    assert np.array_equal(to_host(D), d.astype(np.float64))
    assert np.array_equal(to_host(E), ((T0 - 1.7) - d.astype(np.float64)).astype(np.float32).astype(np.float64))
    back = to_host(api.from_deviation_pair(D, E, 1.7))
    assert np.max(np.abs(back - T0)) <= 2.0 ** -46 * np.max(np.abs(T0))
