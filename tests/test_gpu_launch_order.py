"""Stream order of the step and transposed-step kernels, which are launched with
programmatic dependent launch (a launch may be scheduled while the one before it on
the stream still runs, and waits on griddepcontrol before touching global memory).
Each sequence below interleaves library launches with plain PyTorch kernels that read
and write the same buffers on the same stream - a step reading what a PyTorch kernel
just wrote, a PyTorch kernel overwriting what a step just read, steps that write the
buffer the previous step read - and must give bit for bit the result of the same
sequence with the device synchronized after every operation, and the FP64 oracle's
steps where it applies."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPE = (70, 37, 45)  # nx, ny, nz: several tiles and z-chunks, ragged x and y tails


def setup(scaled):
    """Workload-shaped fields; equal spacings where the coefficient is pre-scaled."""
    T0, Ci, lam, dt, inv = problem(*SHAPE)
    if scaled:
        d = 1.0 / (max(SHAPE) - 1)
        inv = (1.0 / d,) * 3
        dt = d * d / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, inv


def _sequence(T0, Ci, lam, dt, inv, dtype, scaled, sync):
    """Steps with PyTorch kernels in between: T <- step(T) three times, then a
    PyTorch rescale of T (exactly undone later), two more steps, the undo, one step."""
    T = to_dev(T0, dtype)
    C = to_dev(Ci, dtype)
    if scaled:
        C = api.scale_ci(C, lam, dt, inv)
    T2 = torch.empty_like(T)
    api.copy_boundary(T2, T)
    sy = torch.cuda.synchronize if sync else (lambda: None)
    for _ in range(3):
        api.step(T2, T, C, lam, dt, inv, ci_scaled=scaled)
        sy()
        T, T2 = T2, T
    T.mul_(4.0)   # a PyTorch kernel overwrites the field the next step reads
    sy()
    T2.mul_(4.0)  # and the buffer the last step read (its boundary stays consistent)
    sy()
    for _ in range(2):
        api.step(T2, T, C, lam, dt, inv, ci_scaled=scaled)
        sy()
        T, T2 = T2, T
    T.mul_(0.25)
    T2.mul_(0.25)
    sy()
    api.step(T2, T, C, lam, dt, inv, ci_scaled=scaled)
    sy()
    return to_host(T2)


@pytest.mark.parametrize("dtype,scaled", [(torch.float64, True), (torch.float64, False), (torch.float32, False)])
def test_steps_between_pytorch_kernels(dtype, scaled):
    T0, Ci, lam, dt, inv = setup(scaled)
    if dtype == torch.float32:
        T0 = T0 - 1.7  # deviation storage
    free = _sequence(T0, Ci, lam, dt, inv, dtype, scaled, sync=False)
    synced = _sequence(T0, Ci, lam, dt, inv, dtype, scaled, sync=True)
    assert np.array_equal(free, synced)
    if dtype == torch.float64:
        # x4 and x0.25 are exact, and the step is linear in T: six oracle steps
        ref = oracle.run(T0, Ci, lam, dt, *inv, 6)
        assert rel_linf(free, ref) <= 1e-12
    assert api.device_error() == 0


def _adjoint_sequence(Y0, T, Ci, lam, dt, inv, dtype, scaled, sync):
    """Transposed steps ping-ponging ybar / Tbar with a PyTorch kernel between them
    that rewrites the next ybar in place (x2, undone by x0.5 after one more step)."""
    Tt, C = to_dev(T, dtype), to_dev(Ci, dtype)
    if scaled:
        C = api.scale_ci(C, lam, dt, inv)
    y = to_dev(Y0, dtype)
    tb = torch.empty_like(y)
    cb = torch.zeros_like(y)
    sy = torch.cuda.synchronize if sync else (lambda: None)
    for i in range(5):
        api.adjoint(tb, cb, y, Tt, C, lam, dt, inv, ci_scaled=scaled)
        sy()
        y, tb = tb, y
        if i == 1:
            y.mul_(2.0)
            sy()
        if i == 2:
            y.mul_(0.5)
            sy()
    return to_host(y), to_host(cb)


@pytest.mark.parametrize("dtype,scaled", [(torch.float64, True), (torch.float32, False)])
def test_transposed_steps_between_pytorch_kernels(dtype, scaled):
    T0, Ci, lam, dt, inv = setup(scaled)
    rng = np.random.default_rng(3)
    Y0 = rng.standard_normal(T0.shape)
    if dtype == torch.float32:
        T0 = T0 - 1.7
    y_free, c_free = _adjoint_sequence(Y0, T0, Ci, lam, dt, inv, dtype, scaled, sync=False)
    y_sync, c_sync = _adjoint_sequence(Y0, T0, Ci, lam, dt, inv, dtype, scaled, sync=True)
    assert np.array_equal(y_free, y_sync)
    assert np.array_equal(c_free, c_sync)
    assert api.device_error() == 0
