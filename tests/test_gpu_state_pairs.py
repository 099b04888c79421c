"""The FP32 state-keeping loop in fused step pairs (``api.run_states(temporal2=True)``,
``ps_diffusion3d_run_states`` with PS_RUN_TEMPORAL2).  Keeping every state, each pair
writes both states it computes, with their x and y faces; keeping every k-th, a pair
never steps over a kept state.  Every kept grid - boundary included - and T(nt) equal
the one-step loop's states bit for bit; grids the fused-pair kernel cannot serve fall
back to single steps.  The gradient built on these loops equals the one built on single
steps bit for bit."""
import numpy as np
import pytest
import torch

from gpu_helpers import problem, to_dev, to_host
from paper_2211_15634_gb300 import api, autograd
from paper_2211_15634_gb300._lib import PsError

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

# x rows of a multiple of 16 bytes (the fused-pair kernel), ragged x and y tiles, one
# that the TMA kernels cannot serve (odd nx: single column steps), a small grid
SHAPES = [(68, 21, 13), (132, 37, 19), (36, 9, 7), (67, 21, 13), (4, 3, 5)]


def fp32_problem(nx, ny, nz):
    T0h, Ci, lam, dt, inv = problem(nx, ny, nz)
    D0 = to_dev(T0h - 1.7, torch.float32)
    C = to_dev(Ci, torch.float32)
    return D0, C, lam, dt, inv


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("nt,every", [(1, 1), (2, 1), (3, 1), (8, 1), (7, 2), (9, 3), (10, 5), (4, 7)])
@pytest.mark.parametrize("shape", SHAPES)
def test_state_pairs_equal_single_steps(shape, nt, every, graph):
    nx, ny, nz = shape
    D0, C, lam, dt, inv = fp32_problem(nx, ny, nz)
    D0h = to_host(D0)
    block = api.StateBlock(D0, nt // every + (2 if every > 1 else 0), boundary=False)
    block.flat.fill_(float("nan"))  # unprepared grids: the call sets every boundary
    final = api.run_states(D0, block, every, C, lam, dt, inv, nt, graph=graph, temporal2=True)
    a, b = D0.clone(), D0.clone()
    cur = a
    for t in range(1, nt + 1):
        dst = b if cur is a else a
        api.step(dst, cur, C, lam, dt, inv)
        cur = dst
        if t % every == 0:
            assert torch.equal(block.grids[t // every - 1], cur), t
    assert torch.equal(final, cur)
    assert np.array_equal(to_host(D0), D0h)  # T0 is not modified
    api.clear_graph_cache()
    assert api.device_error() == 0


def test_state_pairs_flag_rules():
    """PS_RUN_TEMPORAL2 in the state-keeping loop: FP32 only."""
    nx, ny, nz = 68, 21, 13
    D0, C, lam, dt, inv = fp32_problem(nx, ny, nz)
    T0 = D0.double()
    for every in (1, 2):
        with pytest.raises(PsError):
            api.run_states(T0, api.StateBlock(T0, 4 + 2), every, C.double(), lam, dt, inv, 4, temporal2=True)


@pytest.mark.parametrize("every", [1, 3, 20])
def test_gradient_with_state_pairs_is_bitwise_the_single_step_one(every):
    nx, ny, nz = 68, 21, 13
    nt = 10
    D0, C, lam, dt, inv = fp32_problem(nx, ny, nz)
    Tobs = D0 + 0.01 * torch.sin(torch.arange(D0.numel(), device=D0.device, dtype=torch.float32)).view_as(D0)
    Cg = C * 1.05
    res = [autograd.loss_and_grad(D0, Cg, Tobs, lam, dt, inv, nt, every=every, state_pairs=sp)
           for sp in (False, True)]
    (L0, g0, c0), (L1, g1, c1) = res
    assert torch.equal(L0, L1)
    assert torch.equal(g0, g1)
    assert torch.equal(c0, c1)
    assert torch.count_nonzero(c0) > 0
    assert api.device_error() == 0


def test_state_pairs_at_full_size():
    """512^3 FP32 (the workload's size; 0.5 GiB a state): five states kept, two fused pairs
    that keep both states and one single step, bit for bit the one-step loop's."""
    n, nt = 512, 5
    from paper_2211_15634_gb300 import inputs
    T0 = torch.from_numpy(inputs.t0_gaussian(n, n, n)).cuda()
    D0 = api.to_deviation(T0, 1.7)
    C = api.to_f32(torch.from_numpy(inputs.ci_random(n, n, n)).cuda())
    del T0
    inv = inputs.inverse_spacing(n, n, n)
    dt = api.stable_dt(C, 1.0)
    block = api.StateBlock(D0, nt, boundary=False)
    final = api.run_states(D0, block, 1, C, 1.0, dt, inv, nt, temporal2=True)
    a, b = D0.clone(), D0.clone()
    cur = a
    for t in range(1, nt + 1):
        dst = b if cur is a else a
        api.step(dst, cur, C, 1.0, dt, inv)
        cur = dst
        assert torch.equal(block.grids[t - 1], cur), t
    assert torch.equal(final, cur)
    assert api.device_error() == 0
