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
from paper_2211_15634_gb300 import _lib, api, inputs
from paper_2211_15634_gb300 import autograd as ag

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
def test_adjoint_f32_z_chunks(launch_override, kchunk):
    launch_override(adj_kchunk=kchunk)
    run_case((132, 19, 29))


def test_adjoint_f32_unequal_spacings():
    run_case((136, 21, 18), inv_override=(7.0, 11.0, 5.0))


def test_adjoint_f32_matches_plain_kernel(launch_override):
    """The staged kernel and the plain one-thread-per-column kernel agree to FP32
    rounding on a workload-shaped grid (Gaussian state, random Ci)."""
    nx, ny, nz = 200, 40, 33
    T, Ci, lam, dt, inv = problem(nx, ny, nz)
    ybar = f32(inputs.random_field(T.shape, 9))
    args = [to_dev(f32(a), torch.float32) for a in (ybar, T, Ci)]
    out = []
    for plain in ("0", "1"):
        launch_override(adj_plain=plain)
        Tbar = torch.empty(T.shape, dtype=torch.float32, device="cuda")
        Cib = torch.zeros(T.shape, dtype=torch.float32, device="cuda")
        api.adjoint(Tbar, Cib, *args, lam, dt, inv)
        out.append((to_host(Tbar), to_host(Cib)))
    (ta, ca), (tb, cb) = out
    assert rel_linf(ta, tb) <= TOL
    assert np.max(np.abs(ca - cb)) <= TOL * np.max(np.abs(cb))


# ------------------------------------------------ two transposed steps per pass
def pair_fields(shape, seed=21, inv_override=None):
    nx, ny, nz = shape
    T, Ci, lam, dt, inv = problem(nx, ny, nz, gaussian=False)
    if inv_override is not None:
        inv = inv_override
        dt = 1.0 / (2.0 * sum(v * v for v in inv)) / Ci.max() / 1.05
    S0 = f32(T)
    S1 = f32(T + 0.01 * inputs.random_field(T.shape, seed + 3))
    ybar = f32(inputs.random_field(T.shape, seed))
    cib0 = f32(inputs.random_field(T.shape, seed + 1))
    dev = [to_dev(a, torch.float32) for a in (ybar, S1, S0, f32(Ci), cib0)]
    return dev, lam, dt, inv


@pytest.mark.parametrize("kchunk", ["0", "1", "2", "5"])
@pytest.mark.parametrize("shape", SHAPES + [(136, 21, 18)])
def test_adjoint2_is_two_single_steps(launch_override, kchunk, shape):
    """ps_diffusion3d_adjoint2_ex gives bit for bit two one-step launches (states
    T_first then T_second), Tbar and Cibar, on every grid edge case and z-chunk."""
    launch_override(adj_kchunk=kchunk)
    inv_override = (7.0, 11.0, 5.0) if shape == (136, 21, 18) else None
    (yb, S1, S0, C, cib0), lam, dt, inv = pair_fields(shape, inv_override=inv_override)
    y1 = torch.empty_like(yb)
    tb_ref = torch.empty_like(yb)
    cib_ref = cib0.clone()
    api.adjoint(y1, cib_ref, yb, S1, C, lam, dt, inv)
    api.adjoint(tb_ref, cib_ref, y1, S0, C, lam, dt, inv)
    tb = torch.empty_like(yb)
    cib = cib0.clone()
    api.adjoint2(tb, cib, yb, S1, S0, C, lam, dt, inv)
    assert torch.equal(tb, tb_ref)
    assert torch.equal(cib, cib_ref)
    assert api.device_error() == 0


def test_adjoint2_refusals():
    (yb, S1, S0, C, cib), lam, dt, inv = pair_fields((32, 8, 6))
    tb = torch.empty_like(yb)
    with pytest.raises(_lib.PsError) as e:  # aliasing
        api.adjoint2(yb, cib, yb, S1, S0, C, lam, dt, inv)
    assert e.value.status == _lib.PS_ERR_ALIAS
    d = [t.double() for t in (tb, cib, yb, S1, S0, C)]
    with pytest.raises(_lib.PsError) as e:  # FP64
        api.adjoint2(*d, lam, dt, inv)
    assert e.value.status == _lib.PS_ERR_UNSUPPORTED
    (yb, S1, S0, C, cib), lam, dt, inv = pair_fields((30, 8, 6))
    with pytest.raises(_lib.PsError) as e:  # rows of 120 bytes
        api.adjoint2(torch.empty_like(yb), cib, yb, S1, S0, C, lam, dt, inv)
    assert e.value.status == _lib.PS_ERR_UNSUPPORTED
    assert not api.adjoint2_supported(yb) and api.adjoint2_supported(torch.empty((3, 3, 8)))


@pytest.mark.parametrize("every", [1, 4, None])
def test_fp32_gradient_with_pairs_is_unchanged(every):
    """The reverse sweep in pairs gives bit for bit the sweep one step at a time
    (odd and even segment lengths)."""
    nx, ny, nz, nt = 36, 20, 18, 11
    T0 = inputs.t0_gaussian(nx, ny, nz)
    Ci = inputs.ci_constant(nx, ny, nz) + 0.02 * inputs.random_field((nz, ny, nx), 8)
    Tobs = T0 + 0.01 * inputs.random_field((nz, ny, nx), 9)
    lam = 1.0
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / (1.5 / inputs.C0) / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    D = api.to_deviation(to_dev(T0), 1.7)
    Dobs = api.to_deviation(to_dev(Tobs), 1.7)
    C = api.to_f32(to_dev(Ci))
    a = ag.loss_and_grad(D, C, Dobs, lam, dt, inv, nt, every=every, pairs=False)
    b = ag.loss_and_grad(D, C, Dobs, lam, dt, inv, nt, every=every, pairs=True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
