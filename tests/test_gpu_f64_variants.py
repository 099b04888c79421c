"""The pre-scaled FP64 step at two nodes per thread (launch override ``f64_px2``,
the kernel the library takes when rows do not allow 32-byte accesses) reorganises
the default four-per-thread kernel's per-node arithmetic and must give its result
bit for bit."""
import numpy as np
import pytest
import torch

from gpu_helpers import problem, to_dev, to_host
from paper_2211_15634_gb300 import api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SHAPES = [(64, 9, 7), (132, 21, 17), (68, 40, 11), (256, 35, 19)]


def run(T0, Ci, lam, dt, inv, nt, graph=False):
    T = to_dev(T0)
    C = api.scale_ci(to_dev(Ci), lam, dt, inv)
    return to_host(api.run(T, torch.empty_like(T), C, lam, dt, inv, nt, ci_scaled=True, graph=graph))


def iso(shape):
    T0, Ci, lam, _, _ = problem(*shape)
    d = 1.0 / (max(shape) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, (1.0 / d,) * 3


@pytest.mark.parametrize("shape", SHAPES)
def test_two_per_thread_is_bitwise_equal(launch_override, shape):
    T0, Ci, lam, dt, inv = iso(shape)
    base = run(T0, Ci, lam, dt, inv, 6)
    launch_override(f64_px2=1)
    assert np.array_equal(run(T0, Ci, lam, dt, inv, 6), base)
    assert api.device_error() == 0


def test_px2_override_names_its_kernel(launch_override):
    T = torch.zeros((8, 8, 64), dtype=torch.float64, device="cuda")
    inv = (63.0,) * 3
    assert api.step_kernel_name(T, T.clone(), T.clone(), 1.0, 1e-5, inv, ci_scaled=True) == \
        "k_zmarch<F64_SCALED4>"
    launch_override(f64_px2=1)
    assert api.step_kernel_name(T, T.clone(), T.clone(), 1.0, 1e-5, inv, ci_scaled=True) == \
        "k_zmarch<F64_SCALED>"


def test_graph_replay_across_an_override_change(launch_override):
    """The same buffers run as a cached graph before and after the override changes
    (the change empties the graph cache, so the second run captures the other kernel):
    both equal the plain-stream run bit for bit."""
    T0, Ci, lam, dt, inv = iso((132, 21, 17))
    T, C = to_dev(T0), api.scale_ci(to_dev(Ci), lam, dt, inv)
    T2 = torch.empty_like(T)
    ref = run(T0, Ci, lam, dt, inv, 5)
    outs = []
    for px2 in (0, 1):
        launch_override(f64_px2=px2)
        T.copy_(to_dev(T0))
        outs.append(to_host(api.run(T, T2, C, lam, dt, inv, 5, ci_scaled=True, graph=True)))
    assert np.array_equal(outs[0], ref) and np.array_equal(outs[1], ref)
    api.clear_graph_cache()


def test_graph_cache_is_bounded_and_override_changes_empty_it(launch_override):
    """The graph cache keeps at most 256 graphs (the least recently replayed go first);
    a launch-override change empties it."""
    api.clear_graph_cache()
    T0, Ci, lam, dt, inv = iso((64, 9, 7))
    T, C = to_dev(T0), api.scale_ci(to_dev(Ci), lam, dt, inv)
    T2 = torch.empty_like(T)
    for i in range(300):  # each dt is a new key
        api.run(T, T2, C, lam, dt * (1.0 + 1e-6 * i), inv, 2, ci_scaled=True, graph=True)
    assert api.graph_cache_size() == 256
    torch.cuda.synchronize()
    launch_override(f64_px2=1)
    assert api.graph_cache_size() == 0
    api.run(T, T2, C, lam, dt, inv, 2, ci_scaled=True, graph=True)
    assert api.graph_cache_size() == 1
    api.clear_graph_cache()
