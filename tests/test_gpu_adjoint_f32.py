"""FP32 transposed step (every read staged by TMA) against the FP64 oracle's
adjoint step, over the kernel's tile shapes, z-chunk lengths and grid edges.

Inputs are FP32-representable, so the only difference from the oracle is the
kernel's FP32 rounding: about ten roundings of values bounded by the inputs'
magnitudes, well inside 2e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 2e-6


def f32(a):
    return a.astype(np.float32).astype(np.float64)


def run_case(shape, seed=5, gaussian=False, inv_override=None):
    nx, ny, nz = shape
    T, Ci, lam, dt, inv = problem(nx, ny, nz, gaussian=gaussian)
    if inv_override is not None:
        inv = inv_override
        dt = 1.0 / (2.0 * sum(v * v for v in inv)) / Ci.max() / 1.05
    ybar = inputs.random_field(T.shape, seed)
    cib0 = inputs.random_field(T.shape, seed + 1)
    T, Ci, ybar, cib0 = (f32(a) for a in (T, Ci, ybar, cib0))
    cib_ref = cib0.copy()
    tbar_ref = oracle.adjoint_step(ybar, T, Ci, cib_ref, lam, dt, *inv)
    Tbar = torch.empty(T.shape, dtype=torch.float32, device="cuda")
    Cib = to_dev(cib0, torch.float32)
    api.adjoint(Tbar, Cib, to_dev(ybar, torch.float32), to_dev(T, torch.float32),
                to_dev(Ci, torch.float32), lam, dt, inv)
    got_t, got_c = to_host(Tbar), to_host(Cib)
    assert rel_linf(got_t, tbar_ref) <= TOL
    assert np.max(np.abs(got_c - cib_ref)) <= TOL * np.max(np.abs(cib_ref))
    # boundary entries of Cibar are never written
    inner = np.zeros(T.shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.array_equal(got_c[~inner], cib0[~inner])
    assert api.device_error() == 0


SHAPES = [(4, 5, 6), (8, 3, 3), (132, 19, 13), (256, 9, 17), (260, 37, 41), (128, 16, 3),
          (384, 8, 10)]


@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_f32_grid_edges(shape):
    """Grids smaller than a tile, ragged x-y tiles, several tiles in x, few planes."""
    run_case(shape)


@pytest.mark.parametrize("kchunk", ["1", "2", "3", "7", "64"])
def test_adjoint_f32_z_chunks(monkeypatch, kchunk):
    monkeypatch.setenv("PS_ADJ_KCHUNK", kchunk)
    run_case((132, 19, 29))


def test_adjoint_f32_unequal_spacings():
    run_case((136, 21, 18), inv_override=(7.0, 11.0, 5.0))


def test_adjoint_f32_matches_plain_kernel(monkeypatch):
    """The staged kernel and the plain one-thread-per-column kernel agree to FP32
    rounding on a workload-shaped grid (Gaussian state, random Ci)."""
    nx, ny, nz = 200, 40, 33
    T, Ci, lam, dt, inv = problem(nx, ny, nz)
    ybar = f32(inputs.random_field(T.shape, 9))
    args = [to_dev(f32(a), torch.float32) for a in (ybar, T, Ci)]
    out = []
    for plain in ("0", "1"):
        monkeypatch.setenv("PS_ADJ_PLAIN", plain)
        Tbar = torch.empty(T.shape, dtype=torch.float32, device="cuda")
        Cib = torch.zeros(T.shape, dtype=torch.float32, device="cuda")
        api.adjoint(Tbar, Cib, *args, lam, dt, inv)
        out.append((to_host(Tbar), to_host(Cib)))
    (ta, ca), (tb, cb) = out
    assert rel_linf(ta, tb) <= TOL
    assert np.max(np.abs(ca - cb)) <= TOL * np.max(np.abs(cb))
