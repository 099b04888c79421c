"""The FP64 step's alternative forms selected by PS_F64_VARIANT (measurement
knob): "px2" (pre-scaled step at two nodes per thread instead of four) reorganises
the default kernel's per-node arithmetic and must give its result bit for bit;
"umul" (the step on Ci as given with the coefficient product by a 64 x 64-bit high
multiply and one DFMA) is another rounding of the same step and must meet the FP64
tolerance against the oracle; "by16" is the umul form in 64 x 16 tiles and must
equal umul bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPES = [(64, 9, 7), (132, 21, 17), (68, 40, 11), (256, 35, 19)]


def run(T0, Ci, lam, dt, inv, nt, scaled):
    T = to_dev(T0)
    C = to_dev(Ci)
    if scaled:
        C = api.scale_ci(C, lam, dt, inv)
    return to_host(api.run(T, torch.empty_like(T), C, lam, dt, inv, nt, ci_scaled=scaled))


def iso(shape):
    T0, Ci, lam, _, _ = problem(*shape)
    d = 1.0 / (max(shape) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, (1.0 / d,) * 3


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("base_variant,variant,scaled", [(None, "px2", True), ("umul", "by16", False)])
def test_reorganised_variants_are_bitwise_equal(monkeypatch, shape, base_variant, variant, scaled):
    T0, Ci, lam, dt, inv = iso(shape)
    if base_variant:
        monkeypatch.setenv("PS_F64_VARIANT", base_variant)
    base = run(T0, Ci, lam, dt, inv, 6, scaled)
    monkeypatch.setenv("PS_F64_VARIANT", variant)
    assert np.array_equal(run(T0, Ci, lam, dt, inv, 6, scaled), base)
    assert api.device_error() == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_umul_variant_meets_fp64_tolerance(monkeypatch, shape):
    T0, Ci, lam, dt, inv = iso(shape)
    monkeypatch.setenv("PS_F64_VARIANT", "umul")
    got = run(T0, Ci, lam, dt, inv, 6, False)
    assert rel_linf(got, oracle.run(T0, Ci, lam, dt, *inv, 6)) <= 1e-12
    assert api.device_error() == 0


def test_px2_variant_names_its_kernel(monkeypatch):
    T = torch.zeros((8, 8, 64), dtype=torch.float64, device="cuda")
    inv = (63.0,) * 3
    assert api.step_kernel_name(T, T.clone(), T.clone(), 1.0, 1e-5, inv, ci_scaled=True) == \
        "k_zmarch<F64_SCALED4>"
    monkeypatch.setenv("PS_F64_VARIANT", "px2")
    assert api.step_kernel_name(T, T.clone(), T.clone(), 1.0, 1e-5, inv, ci_scaled=True) == \
        "k_zmarch<F64_SCALED>"
