"""2-D form of the step (Fig. 1's step! with the z term dropped) on the GPU against
the pinned 2-D oracle: FP64 (pre-scaled coefficient, the emulated step on Ci as
given, plain FP64 for unequal spacings) and FP32 in deviation storage, edge cases
of the warp strips and row chunks, the graph-captured loop."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FP64_TOL = 1e-12
U32 = 2.0 ** -24


def fields2d(nx, ny, seed=7, equal=True, gaussian=True):
    Ci = inputs.ci_random(nx, ny, 1, seed=seed)[0]
    if gaussian:
        x = np.arange(nx) / (nx - 1)
        y = np.arange(ny) / (ny - 1)
        T0 = 1.7 + np.exp(-((x[None, :] - 0.5) ** 2 + (y[:, None] - 0.5) ** 2) / 0.01)
    else:
        T0 = 1.7 + inputs.random_field((ny, nx), seed + 1, 0.0, 1.0)
    if equal:
        d = 1.0 / (max(nx, ny) - 1)
        dx = dy = d
    else:
        dx, dy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    dt = min(dx * dx, dy * dy) / Ci.max() / 4.1
    return np.ascontiguousarray(T0), Ci, dt, (1.0 / dx, 1.0 / dy)


def gpu_run2d(T0, Ci, dt, inv, nt, dtype=torch.float64, **kw):
    T = to_dev(T0, dtype)
    return to_host(api.run2d(T, torch.empty_like(T), to_dev(Ci, dtype), 1.0, dt, inv, nt, **kw))


SHAPES = [(3, 3), (4, 5), (5, 4), (33, 17), (64, 40), (66, 9), (130, 70), (257, 129), (1000, 37), (36, 300)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nt", [1, 6])
def test_fp64_matches_oracle(shape, nt):
    nx, ny = shape
    T0, Ci, dt, inv = fields2d(nx, ny, gaussian=False)
    ref = oracle.run2d(T0, Ci, 1.0, dt, *inv, nt)
    assert rel_linf(gpu_run2d(T0, Ci, dt, inv, nt), ref) <= FP64_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_unequal_spacings_match_oracle(shape):
    nx, ny = shape
    T0, Ci, dt, inv = fields2d(nx, ny, equal=False, gaussian=False)
    ref = oracle.run2d(T0, Ci, 1.0, dt, *inv, 5)
    assert rel_linf(gpu_run2d(T0, Ci, dt, inv, 5), ref) <= FP64_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_prescaled_matches_oracle(shape):
    nx, ny = shape
    T0, Ci, dt, inv = fields2d(nx, ny)
    nt = 7
    ref = oracle.run2d(T0, Ci, 1.0, dt, *inv, nt)
    Cs = api.scale_ci(to_dev(Ci), 1.0, dt, inv)
    T = to_dev(T0)
    got = to_host(api.run2d(T, torch.empty_like(T), Cs, 1.0, dt, inv, nt, ci_scaled=True))
    assert rel_linf(got, ref) <= FP64_TOL


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_deviation_matches_oracle(shape):
    nx, ny = shape
    T0, Ci, dt, inv = fields2d(nx, ny)
    D0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
    C32 = Ci.astype(np.float32).astype(np.float64)
    nt = 6
    ref = oracle.run2d(D0, C32, 1.0, dt, *inv, nt)
    got = gpu_run2d(D0, C32, dt, inv, nt, dtype=torch.float32)
    assert np.max(np.abs(got - ref)) <= nt * 13 * U32 * np.max(np.abs(D0)) + 1e-30


@pytest.mark.parametrize("chunk", ["1", "3", "16", "300"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_row_chunks_do_not_change_results(launch_override, chunk, dtype):
    T0, Ci, dt, inv = fields2d(130, 77, gaussian=False)
    base = gpu_run2d(T0, Ci, dt, inv, 4, dtype=dtype)
    launch_override(chunk2d=chunk)
    assert np.array_equal(gpu_run2d(T0, Ci, dt, inv, 4, dtype=dtype), base)


def test_graph_equals_stream_and_edges_are_kept():
    T0, Ci, dt, inv = fields2d(200, 150, gaussian=False)
    a = gpu_run2d(T0, Ci, dt, inv, 9, graph=True)
    b = gpu_run2d(T0, Ci, dt, inv, 9, graph=False)
    assert np.array_equal(a, b)
    edge = np.ones(T0.shape, dtype=bool)
    edge[1:-1, 1:-1] = False
    assert np.array_equal(a[edge], T0[edge])
    api.clear_graph_cache()


def test_step_writes_interior_only():
    T0, Ci, dt, inv = fields2d(67, 33, gaussian=False)
    T = to_dev(T0)
    T2 = torch.full_like(T, -5.0)
    api.step2d(T2, T, to_dev(Ci), 1.0, dt, inv)
    out = to_host(T2)
    inner = np.zeros(T0.shape, dtype=bool)
    inner[1:-1, 1:-1] = True
    assert np.all(out[~inner] == -5.0)
    ref = np.full_like(T0, -5.0)
    oracle.step2d(ref, T0, Ci, 1.0, dt, *inv)
    assert rel_linf(out[inner], ref[inner]) <= 1e-15


@pytest.mark.parametrize("shape,lengths,dtype", [((130, 70), (1.0, 1.0), torch.float64),
                                                 ((33, 170), (2.0, 0.5), torch.float64),
                                                 ((64, 64), (1.0, 1.0), torch.float32)])
def test_stable_dt2d_matches_oracle(shape, lengths, dtype):
    """ps_diffusion2d_stable_dt (maximum on the GPU, dt formed in the library) equals
    the oracle's 2-D dt bit for bit; FP32 fields reduce their FP32 values."""
    nx, ny = shape
    Ci = inputs.ci_random(nx, ny, 1, seed=3)[0]
    if dtype == torch.float32:
        Ci = Ci.astype(np.float32).astype(np.float64)
    lam = 0.9
    dx, dy = lengths[0] / (nx - 1), lengths[1] / (ny - 1)
    ref = oracle.stable_dt2d(dx, dy, lam, oracle.maximum(Ci))
    assert api.stable_dt2d(to_dev(Ci, dtype), lam, lengths) == ref


N2_BIG = 46368  # 46368^2 = 2,149,991,424 nodes > 2^31


def test_fp64_2d_past_2e31_elements():
    """The 2-D form at 46368^2 FP64 (element offsets past 2^31, 17 GB a field), pre-scaled
    coefficient, nt = 2: sampled nodes - interior, edges, corners' neighbours - against the
    2-D oracle on each sample's dependency cone, whose inputs come from the same
    counter-based draws on the host."""
    n, nt = N2_BIG, 2
    dev = torch.device("cuda")
    T = torch.empty((n, n), dtype=torch.float64, device=dev)
    C = torch.empty_like(T)
    for j0 in range(0, n, 4096):  # the draws a slab of rows at a time (bounded temporaries)
        j1 = min(n, j0 + 4096)
        idx = torch.arange(j0 * n, j1 * n, dtype=torch.int64, device=dev)
        T[j0:j1] = (inputs.T_BASE + inputs.uniform_torch(99, idx)).view(j1 - j0, n)
        C[j0:j1] = (((inputs.uniform_torch(inputs.SEED_CI, idx) * 0.5) + 1.0) * (1.0 / inputs.C0)).view(j1 - j0, n)
    assert T.numel() > 2 ** 31
    dt = api.stable_dt2d(C, 1.0)
    inv = (float(n - 1), float(n - 1))
    api.scale_ci(C, 1.0, dt, inv, out=C)  # in place: Cs
    res = api.run2d(T, torch.empty_like(T), C, 1.0, dt, inv, nt, ci_scaled=True)
    pts = [(n // 2, n // 2), (1, 1), (n - 2, n - 3), (0, 4000), (n - 1, 45000), (30000, n - 2), (46000, 2)]
    jj = torch.tensor([p[1] for p in pts], device=dev)
    ii = torch.tensor([p[0] for p in pts], device=dev)
    got = res[jj, ii].cpu().numpy()
    ref = []
    for (i, j) in pts:
        i0, i1 = max(0, i - nt), min(n, i + nt + 1)
        j0, j1 = max(0, j - nt), min(n, j + nt + 1)
        J, I = np.meshgrid(np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
        idx = (I + n * J).astype(np.uint64)
        T0c = inputs.T_BASE + inputs.uniform(99, idx)
        Cic = ((inputs.uniform(inputs.SEED_CI, idx) * 0.5) + 1.0) * (1.0 / inputs.C0)
        out = oracle.run2d(T0c, Cic, 1.0, dt, *inv, nt) if min(T0c.shape) >= 3 else T0c
        ref.append(out[j - j0, i - i0])
    assert np.max(np.abs(got - np.array(ref))) <= FP64_TOL * 2.7
    assert api.device_error() == 0
    del T, C, res
    torch.cuda.empty_cache()
