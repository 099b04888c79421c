"""The FP64 step's paths for warps whose values leave one binade: the window path
(values of one sign within five adjacent binades: cheap exact integer sums) and the
general fixed-point path (each node's values at 57 bits below its largest exponent:
exact within five binades, low-order bits of smaller values dropped beyond).  Both
are deterministic node by node, so the z-march step must give bit for bit the
per-node general arithmetic of the kernels that step node by node:
the fused-pair kernel (pre-scaled coefficient) and the column kernel (Ci as given,
forced by the step_plain launch override), and the FP64 oracle within 1e-12."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPE = (132, 21, 17)


def field(kind, shape=SHAPE, seed=11):
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = inputs.random_field((nz, ny, nx), seed, 0.0, 1.0)
    if kind == "two_binades":  # every stencil straddles 1.0: binades [0.5, 1) and [1, 2)
        return 1.0 + 0.05 * np.where((i + j + k) % 2 == 0, 1.0, -1.0) * (1.0 + 0.1 * r)
    if kind == "two_binades_negative":
        return -field("two_binades", shape, seed)
    if kind == "window":  # one sign, seven binades: lanes in five take the window path, others not
        return np.exp2(6.0 * r) * (1.0 + 0.5 * np.where((i + j + k) % 2 == 0, 1.0, -1.0) * r)
    if kind == "window_negative":
        return -field("window", shape, seed)
    if kind == "many_binades":  # signs, zeros and tiny values: the general path
        T = 2.0 * r - 1.0
        T[::3, :, ::5] = 0.0
        T[1::4, ::2, :] *= 1e-9
        return T
    raise ValueError(kind)


def setup(kind):
    nx, ny, nz = SHAPE
    T0 = field(kind)
    Ci = inputs.ci_random(nx, ny, nz)
    d = 1.0 / (max(SHAPE) - 1)
    dt = d * d / Ci.max() / 6.1
    return T0, Ci, dt, (1.0 / d,) * 3


KINDS = ["two_binades", "two_binades_negative", "window", "window_negative", "many_binades"]


@pytest.mark.parametrize("kind", KINDS)
def test_prescaled_step_equals_per_node_pairs(kind):
    """Pre-scaled coefficient: nt single z-march steps = nt/2 fused pairs (the pair
    kernel steps node by node) bit for bit, and the oracle within 1e-12."""
    T0, Ci, dt, inv = setup(kind)
    C = api.scale_ci(to_dev(Ci), 1.0, dt, inv)
    nt = 4
    runs = []
    for t2 in (False, True):
        T = to_dev(T0)
        runs.append(to_host(api.run(T, torch.empty_like(T), C, 1.0, dt, inv, nt, ci_scaled=True,
                                    temporal2=t2)))
    assert np.array_equal(runs[0], runs[1])
    assert rel_linf(runs[0], oracle.run(T0, Ci, 1.0, dt, *inv, nt)) <= 1e-12
    assert api.device_error() == 0


@pytest.mark.parametrize("kind", KINDS)
def test_ci_as_given_step_equals_column_kernel(launch_override, kind):
    """Ci as given: on fields where every warp leaves one binade, the z-march step
    equals the column kernel's per-node arithmetic bit for bit (a warp whose values
    all share one binade would take the z-march's own one-binade form, fma(Ci*K, S, T),
    which rounds differently; none does on these fields)."""
    T0, Ci, dt, inv = setup(kind)
    nt = 3
    runs = []
    for plain in (0, 1):
        launch_override(step_plain=plain)
        T = to_dev(T0)
        runs.append(to_host(api.run(T, torch.empty_like(T), to_dev(Ci), 1.0, dt, inv, nt)))
    ref = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
    assert rel_linf(runs[0], ref) <= 1e-12
    assert np.array_equal(runs[0], runs[1])
