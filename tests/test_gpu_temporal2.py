"""Two steps per pass (PS_RUN_TEMPORAL2): the fused pairs give bit for bit the
states of single steps (the same per-node arithmetic), so the time loop is
compared with the one-step loop exactly and with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import _lib, api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def iso_problem(nx, ny, nz, gaussian=False):
    T0 = inputs.t0_gaussian(nx, ny, nz) if gaussian else \
        1.7 + inputs.random_field((nz, ny, nx), 99, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    lam = 1.0
    d = 1.0 / (max(nx, ny, nz) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, (1.0 / d,) * 3


def run64(T0, Ci, lam, dt, inv, nt, **kw):
    T = to_dev(T0)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    return to_host(api.run(T, torch.empty_like(T), Cs, lam, dt, inv, nt, ci_scaled=True, **kw))


def run32(D0, C, lam, dt, inv, nt, **kw):
    D = to_dev(D0, torch.float32)
    return to_host(api.run(D, torch.empty_like(D), to_dev(C, torch.float32), lam, dt, inv, nt, **kw))


SHAPES = [(4, 5, 6), (64, 8, 9), (66, 19, 20), (132, 21, 17), (130, 67, 33), (256, 35, 19),
          (68, 70, 40), (200, 3, 4)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nt", [1, 2, 3, 6, 9])
def test_fp64_pairs_equal_single_steps_and_oracle(shape, nt):
    T0, Ci, lam, dt, inv = iso_problem(*shape)
    one = run64(T0, Ci, lam, dt, inv, nt)
    two = run64(T0, Ci, lam, dt, inv, nt, temporal2=True)
    assert np.array_equal(one, two)
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    assert rel_linf(two, ref) <= 1e-12
    assert api.device_error() == 0


@pytest.mark.parametrize("shape", [(4, 5, 6), (132, 21, 17), (256, 35, 19), (68, 70, 40)])
@pytest.mark.parametrize("nt", [2, 5, 8])
def test_fp32_pairs_equal_single_steps(shape, nt):
    nx, ny, nz = shape
    T0, Ci, lam, _, _ = iso_problem(nx, ny, nz)
    dx, dy, dz = inputs.spacing(nx, ny, nz)  # anisotropic spacings are fine in FP32
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci.max() / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    D0 = T0 - 1.7
    one = run32(D0, Ci, lam, dt, inv, nt)
    two = run32(D0, Ci, lam, dt, inv, nt, temporal2=True)
    assert np.array_equal(one, two)
    assert api.device_error() == 0


@pytest.mark.parametrize("kchunk", ["1", "2", "5", "40"])
def test_pairs_short_and_long_z_chunks(launch_override, kchunk):
    launch_override(kchunk2=kchunk)
    T0, Ci, lam, dt, inv = iso_problem(136, 27, 22, gaussian=True)
    one = run64(T0, Ci, lam, dt, inv, 6)
    assert np.array_equal(one, run64(T0, Ci, lam, dt, inv, 6, temporal2=True))
    D0 = T0 - 1.7
    assert np.array_equal(run32(D0, Ci, lam, dt, inv, 6),
                          run32(D0, Ci, lam, dt, inv, 6, temporal2=True))
    assert api.device_error() == 0


def test_pairs_general_path_graph_and_kernel_name():
    """Signs and binade changes (fixed-point general path) through the fused
    kernel, replayed as a CUDA graph."""
    nx, ny, nz, nt = 64, 31, 17, 8
    _, Ci, lam, dt, inv = iso_problem(nx, ny, nz)
    T0 = inputs.random_field((nz, ny, nx), 78, -1.0, 1.0)
    T0[::3, :, ::5] = 0.0
    T0[1::4, ::2, :] *= 1e-9
    one = run64(T0, Ci, lam, dt, inv, nt)
    assert np.array_equal(one, run64(T0, Ci, lam, dt, inv, nt, temporal2=True))
    assert np.array_equal(one, run64(T0, Ci, lam, dt, inv, nt, temporal2=True, graph=True))
    api.clear_graph_cache()
    T = to_dev(T0)
    Cs = api.scale_ci(to_dev(Ci), lam, dt, inv)
    assert api.step_kernel_name(torch.empty_like(T), T, Cs, lam, dt, inv, ci_scaled=True,
                                temporal2=True) == "k_zmarch2<F64_SCALED>"


def test_pairs_fall_back_on_odd_nx_and_reject_other_modes():
    T0, Ci, lam, dt, inv = iso_problem(37, 29, 23)  # nx*8 not a multiple of 16: single steps
    assert np.array_equal(run64(T0, Ci, lam, dt, inv, 4), run64(T0, Ci, lam, dt, inv, 4, temporal2=True))
    T = to_dev(T0)
    with pytest.raises(_lib.PsError, match="TEMPORAL2"):
        api.run(T, torch.empty_like(T), to_dev(Ci), lam, dt, inv, 4, temporal2=True)  # FP64 on Ci
    D = to_dev(T0 - 1.7, torch.float32)
    with pytest.raises(_lib.PsError, match="TEMPORAL2"):
        api.run(D, torch.empty_like(D), to_dev(Ci, torch.float32), lam, dt, inv, 4,
                comp=api.compensation_fields(D), temporal2=True)
