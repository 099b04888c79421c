"""Full-size parity in the launch configurations bench.py times, on outputs the
oracle can compute one by one (each sampled node from its dependency cone) or,
for the batch, on whole problems.

* FP64 512^3, nt = 100: dt from maximum(Ci) on the GPU, the pre-scaled
  coefficient, the graph-captured loop of the TMA step (the headline path).
* FP32 1024^3, nt = 100, deviation storage (the bench's FP32 1024^3 row), and the
  compensated two-float step at 512^3 (the bench's compensated row).
* The 256-problem batch, nt = 500, padded rows, the TMA z-march with tuned
  z-chunks (FP64 on the pre-scaled coefficient, and FP32): the smallest
  problems and the largest one against the oracle's own runs.
* FP64 768^3 (byte offsets past 2^32), sampled like 512^3.
* FP64 and FP32 1296^3: 2,176,782,336 nodes, element offsets past 2^31 (fields made
  on the device from the same counter-based draws the host uses for the samples'
  cones), dt from maximum(Ci) over the whole field.
* The gradient workload (256^3, nt = 200, FP64): directional derivatives of the
  adjoint against central differences of FP64 forward runs, to 1e-6.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
from gpu_helpers import light_cone_reference, problem, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs, tuner

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FP64_TOL = 1e-12
U32 = 2.0 ** -24


def sample(t: torch.Tensor, pts):
    """Values of a device field at nodes (i, j, k), gathered on the device."""
    k = torch.tensor([p[2] for p in pts], device=t.device)
    j = torch.tensor([p[1] for p in pts], device=t.device)
    i = torch.tensor([p[0] for p in pts], device=t.device)
    return t[k, j, i].double().cpu().numpy()


PTS512 = [(256, 256, 256), (1, 1, 1), (510, 300, 7), (255, 3, 509), (120, 400, 256), (0, 17, 30)]


def test_fp64_512_bench_path():
    n, nt = 512, 100
    T0, Ci, inv = bench.fields(n)
    dev = torch.device("cuda")
    T = torch.from_numpy(T0).to(dev)
    C = torch.from_numpy(Ci).to(dev)
    dt = api.stable_dt(C, 1.0)
    assert dt == oracle.stable_dt(1 / (n - 1), 1 / (n - 1), 1 / (n - 1), 1.0, oracle.maximum(Ci))
    Cs = api.scale_ci(C, 1.0, dt, inv)
    assert api.step_kernel_name(T, T, Cs, 1.0, dt, inv, ci_scaled=True) == "k_zmarch<F64_SCALED4>"
    res = api.run(T, torch.empty_like(T), Cs, 1.0, dt, inv, nt, graph=True, ci_scaled=True)
    got = sample(res, PTS512)
    oracle.set_threads(max(1, oracle.max_threads()))
    try:
        ref = light_cone_reference(oracle, T0, Ci, 1.0, dt, inv, nt, PTS512)
    finally:
        oracle.set_threads(1)
    assert np.max(np.abs(got - ref)) <= FP64_TOL * np.max(np.abs(T0))
    assert float(res.min()) >= T0.min() - 1e-12 and float(res.max()) <= T0.max() + 1e-12
    assert api.device_error() == 0
    api.clear_graph_cache()


def test_fp32_compensated_512_bench_path():
    """The bench's compensated FP32 row (512^3, nt = 100, graph) from the two-float
    deviation of T0: sampled nodes against the oracle on the same starting state and
    the FP32 Ci: within 2e-8 of max|D0|, ten times the compensated arithmetic error the
    bench measures at 256^3 and far inside the plain FP32 bound (7.7e-5 here)."""
    n, nt = 512, 100
    T0, Ci, inv = bench.fields(n)
    dev = torch.device("cuda")
    D, E0 = api.to_deviation_pair(torch.from_numpy(T0).to(dev), 1.7)
    C32 = api.to_f32(torch.from_numpy(Ci).to(dev))
    dt = api.stable_dt(C32, 1.0)
    comp = api.compensation_fields(D, E0)
    start = api.from_deviation_pair(D, E0, 0.0).cpu().numpy()
    res = api.run(D, torch.empty_like(D), C32, 1.0, dt, inv, nt, comp=comp, graph=True)
    got = sample(api.from_deviation_pair(res, comp[nt % 2], 0.0), PTS512)
    C0 = Ci.astype(np.float32).astype(np.float64)
    oracle.set_threads(max(1, oracle.max_threads()))
    try:
        ref = light_cone_reference(oracle, start, C0, 1.0, dt, inv, nt, PTS512)
    finally:
        oracle.set_threads(1)
    assert np.max(np.abs(got - ref)) <= 2e-8 * np.max(np.abs(start))
    assert api.device_error() == 0
    api.clear_graph_cache()


PTS1024 = [(512, 512, 512), (1, 1022, 3), (1000, 40, 700), (300, 800, 1022)]


def test_fp32_1024_bench_path():
    n, nt = 1024, 100
    T0, Ci, inv = bench.fields(n)
    dev = torch.device("cuda")
    D = api.to_deviation(torch.from_numpy(T0).to(dev), 1.7)
    C32 = api.to_f32(torch.from_numpy(Ci).to(dev))
    dt = api.stable_dt(C32, 1.0)
    res = api.run(D, torch.empty_like(D), C32, 1.0, dt, inv, nt, graph=True)
    got = sample(res, PTS1024)
    # the oracle on the FP32-rounded inputs, on each sample's cone only
    D0 = (T0 - 1.7).astype(np.float32).astype(np.float64)
    C0 = Ci.astype(np.float32).astype(np.float64)
    oracle.set_threads(max(1, oracle.max_threads()))
    try:
        ref = light_cone_reference(oracle, D0, C0, 1.0, dt, inv, nt, PTS1024)
    finally:
        oracle.set_threads(1)
    assert np.max(np.abs(got - ref)) <= nt * 13 * U32 * np.max(np.abs(D0))
    api.clear_graph_cache()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_256_bench_path(tmp_path, monkeypatch, dtype):
    monkeypatch.setenv("PS_TUNER_CACHE", str(tmp_path / "tuner.json"))
    nt = 500
    dev = torch.device("cuda")
    scaled = dtype == torch.float64
    probs, _ = bench.batch_workload(torch, api, inputs, dtype, dev, 256, pitched=True, ci_scaled=scaled)
    sizes = [int(p["T"].shape[0]) for p in probs]
    b = tuner.tuned_batch(probs, kernel="zmarch", ci_scaled=scaled)  # as the bench runs it
    # the tuner stepped the fields: start again from T0
    order = np.argsort(sizes)
    check = [int(q) for q in order[:3]] + [int(order[-1])]
    for q, p in enumerate(probs):
        T0q, _ = inputs.batch_problem(q, sizes[q])
        Tq = torch.from_numpy(T0q).to(dev)
        if dtype == torch.float32:
            Tq = api.to_deviation(Tq, 1.7)
        p["T"].copy_(Tq)
        p["T2"].copy_(Tq)
    b.run(nt, graph=True)
    oracle.set_threads(max(1, oracle.max_threads()))
    try:
        for q in check:
            n = sizes[q]
            T0q, Ciq = inputs.batch_problem(q, n)
            dtq = probs[q]["dt"]
            inv = inputs.inverse_spacing(n, n, n)
            got = to_host(b.result(q, nt))
            if dtype == torch.float64:
                ref = oracle.run(T0q, Ciq, 1.0, dtq, *inv, nt)
                assert np.max(np.abs(got - ref)) <= FP64_TOL * np.max(np.abs(ref)), (q, n)
            else:
                D0 = (T0q - 1.7).astype(np.float32).astype(np.float64)
                C0 = Ciq.astype(np.float32).astype(np.float64)
                ref = oracle.run(D0, C0, 1.0, dtq, *inv, nt)
                assert np.max(np.abs(got - ref)) <= nt * 13 * U32 * np.max(np.abs(D0)), (q, n)
    finally:
        oracle.set_threads(1)
    assert api.device_error() == 0
    api.clear_graph_cache()


def test_fp64_768_bench_path():
    """The bench's 768^3 FP64 row (3.4 GiB per field: byte offsets past 2^32)."""
    n, nt = 768, 100
    T0, Ci, inv = bench.fields(n)
    dev = torch.device("cuda")
    T = torch.from_numpy(T0).to(dev)
    C = torch.from_numpy(Ci).to(dev)
    dt = api.stable_dt(C, 1.0)
    Cs = api.scale_ci(C, 1.0, dt, inv)
    res = api.run(T, torch.empty_like(T), Cs, 1.0, dt, inv, nt, graph=True, ci_scaled=True)
    pts = [(384, 384, 384), (766, 1, 500), (2, 700, 766), (700, 5, 3)]
    got = sample(res, pts)
    oracle.set_threads(max(1, oracle.max_threads()))
    try:
        ref = light_cone_reference(oracle, T0, Ci, 1.0, dt, inv, nt, pts)
    finally:
        oracle.set_threads(1)
    assert np.max(np.abs(got - ref)) <= FP64_TOL * np.max(np.abs(T0))
    api.clear_graph_cache()


@pytest.mark.parametrize("every", [15, 1])  # ceil(sqrt(200)) and every state kept
def test_gradient_256_directional_derivatives(every):
    """The bench's gradient workload (256^3, nt = 200, FP64, sqrt(nt) checkpoints or
    every state kept): the adjoint's directional derivatives in T0 and Ci against
    central differences of the loss computed by FP64 forward runs.  L is exactly
    quadratic in T0 (the central difference is exact up to rounding); in Ci the
    difference error is O(h^2)."""
    from paper_2211_15634_gb300 import autograd as ag
    n, nt = 256, 200
    dev = torch.device("cuda")
    T0 = torch.from_numpy(inputs.t0_gaussian(n, n, n)).to(dev)
    inv = inputs.inverse_spacing(n, n, n)
    dx = 1.0 / (n - 1)
    dt = dx * dx / 1.0 / (1.5 / inputs.C0) / 6.1
    Ct = torch.from_numpy(inputs.ci_smooth(n, n, n)).to(dev)
    Tobs = api.run(T0.clone(), T0.clone(), Ct, 1.0, dt, inv, nt).clone()
    Ci = torch.full_like(T0, 1.0 / inputs.C0) + 0.02 * torch.from_numpy(
        inputs.random_field((n, n, n), 8)).to(dev)
    L, dT0, dCi = ag.loss_and_grad(T0, Ci, Tobs, 1.0, dt, inv, nt, every=every)

    def loss(T0_, Ci_):
        out = api.run(T0_.clone(), T0_.clone(), Ci_, 1.0, dt, inv, nt)
        return float(api.half_sq_dist(out, Tobs))

    assert abs(loss(T0, Ci) - float(L)) <= 1e-12 * float(L)
    v = torch.from_numpy(inputs.random_field((n, n, n), 11)).to(dev)
    v[0, :, :] = v[-1, :, :] = v[:, 0, :] = v[:, -1, :] = v[:, :, 0] = v[:, :, -1] = 0.0
    h = 1e-4
    fd = (loss(T0, Ci + h * v) - loss(T0, Ci - h * v)) / (2 * h)
    ad = float(api.dot(dCi, v))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    w = torch.from_numpy(inputs.random_field((n, n, n), 12)).to(dev)
    h = 1e-3
    fd = (loss(T0 + h * w, Ci) - loss(T0 - h * w, Ci)) / (2 * h)
    ad = float(api.dot(dT0, w))
    assert abs(fd - ad) <= 1e-6 * abs(ad)


# ------------------------------------------------------- past 2^31 elements
N_BIG = 1296  # 1296^3 = 2,176,782,336 nodes > 2^31 = 2,147,483,648
PTS_BIG = [(648, 648, 648), (1294, 1294, 1294), (3, 1200, 1279), (1000, 5, 1294), (1295, 600, 1285),
           (700, 1293, 1280)]
SEED_T_BIG = 99


def big_fields(dev):
    """T0 = 1.7 + U (seed 99) and the workload's Ci on the 1296^3 grid, made on the device
    from the counter-based draws (inputs.uniform_field_torch)."""
    n = N_BIG
    T = inputs.uniform_field_torch(SEED_T_BIG, n, n, n, dev)
    T += inputs.T_BASE
    C = inputs.uniform_field_torch(inputs.SEED_CI, n, n, n, dev)
    C.mul_(0.5).add_(1.0).mul_(1.0 / inputs.C0)
    return T, C


def big_cones(pts, nt):
    """(T0, Ci) on each sample's dependency cone, from the same draws on the host."""
    n = N_BIG
    out = []
    for (i, j, k) in pts:
        i0, i1 = max(0, i - nt), min(n, i + nt + 1)
        j0, j1 = max(0, j - nt), min(n, j + nt + 1)
        k0, k1 = max(0, k - nt), min(n, k + nt + 1)
        kk, jj, ii = np.meshgrid(np.arange(k0, k1), np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
        idx = (ii + n * (jj + n * kk)).astype(np.uint64)
        T0 = inputs.T_BASE + inputs.uniform(SEED_T_BIG, idx)
        u = inputs.uniform(inputs.SEED_CI, idx)
        Ci = ((u * 0.5) + 1.0) * (1.0 / inputs.C0)
        out.append(((i - i0, j - j0, k - k0), T0, Ci))
    return out


def cone_refs(cones, lam, dt, inv, nt):
    """The oracle's T(nt) at each sample, run on its cone (a cone thinner than three
    nodes holds a boundary sample, which keeps its value)."""
    ref = []
    for (li, lj, lk), T0, Ci in cones:
        res = oracle.run(T0, Ci, lam, dt, *inv, nt) if min(T0.shape) >= 3 else T0
        ref.append(res[lk, lj, li])
    return np.array(ref)


def test_fp64_past_2e31_elements():
    n, nt = N_BIG, 2
    dev = torch.device("cuda")
    T, C = big_fields(dev)
    assert T.numel() > 2 ** 31
    cones = big_cones(PTS_BIG, nt)
    # the cones' inputs are the device fields' values (same draws, same operations)
    for (pt, (_, T0c, Cic)) in zip(PTS_BIG, cones):
        i, j, k = pt
        assert T0c[min(k, nt), min(j, nt), min(i, nt)] == float(T[k, j, i])
        assert Cic[min(k, nt), min(j, nt), min(i, nt)] == float(C[k, j, i])
    assert api.maximum(C) == float(C.max())  # the reduction over the whole field
    dt = api.stable_dt(C, 1.0)
    inv = inputs.inverse_spacing(n, n, n)
    api.scale_ci(C, 1.0, dt, inv, out=C)  # in place: Cs
    T2 = torch.empty_like(T)
    res = api.run(T, T2, C, 1.0, dt, inv, nt, ci_scaled=True)
    got = sample(res, PTS_BIG)
    ref = cone_refs(cones, 1.0, dt, inv, nt)
    assert np.max(np.abs(got - ref)) <= FP64_TOL * 2.7
    assert api.device_error() == 0
    del T, T2, C, res
    torch.cuda.empty_cache()


def test_fp32_past_2e31_elements():
    n, nt = N_BIG, 2
    dev = torch.device("cuda")
    D = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    C32 = torch.empty_like(D)
    for k0 in range(0, n, 64):  # FP64 draws a slab at a time, rounded to FP32 like the host
        k1 = min(n, k0 + 64)
        idx = torch.arange(k0 * n * n, k1 * n * n, dtype=torch.int64, device=dev)
        D[k0:k1] = ((inputs.T_BASE + inputs.uniform_torch(SEED_T_BIG, idx)) - inputs.T_BASE).view(k1 - k0, n, n)
        u = inputs.uniform_torch(inputs.SEED_CI, idx)
        C32[k0:k1] = (((u * 0.5) + 1.0) * (1.0 / inputs.C0)).view(k1 - k0, n, n)
    dt = api.stable_dt(C32, 1.0)
    inv = inputs.inverse_spacing(n, n, n)
    res = api.run(D, torch.empty_like(D), C32, 1.0, dt, inv, nt)
    got = sample(res, PTS_BIG)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    cones = [(loc, f32(T0 - inputs.T_BASE), f32(Ci)) for loc, T0, Ci in big_cones(PTS_BIG, nt)]
    ref = cone_refs(cones, 1.0, dt, inv, nt)
    assert np.max(np.abs(got - ref)) <= nt * 13 * U32 * 1.0
    assert api.device_error() == 0
    del D, C32, res
    torch.cuda.empty_cache()


SEED_YBAR_BIG = 77


def adjoint_blocks(pts, n):
    """(ybar, T, Ci) on the 5^3 block around each sample (clipped at the domain), from the
    host draws: the sample's transposed step reads w and T at its six neighbours, which
    are interior nodes of the block exactly when they are interior nodes of the grid."""
    out = []
    for (i, j, k) in pts:
        i0, i1 = max(0, i - 2), min(n, i + 3)
        j0, j1 = max(0, j - 2), min(n, j + 3)
        k0, k1 = max(0, k - 2), min(n, k + 3)
        kk, jj, ii = np.meshgrid(np.arange(k0, k1), np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
        idx = (ii + n * (jj + n * kk)).astype(np.uint64)
        T = inputs.T_BASE + inputs.uniform(SEED_T_BIG, idx)
        Ci = ((inputs.uniform(inputs.SEED_CI, idx) * 0.5) + 1.0) * (1.0 / inputs.C0)
        ybar = inputs.uniform(SEED_YBAR_BIG, idx) - 0.5
        out.append(((i - i0, j - j0, k - k0), ybar, T, Ci))
    return out


def adjoint_refs(blocks, lam, dt, inv, cast=None):
    """The oracle's transposed step (Tbar, dL/dCi term) at each block's sample."""
    tb, cb = [], []
    for (li, lj, lk), ybar, T, Ci in blocks:
        if cast is not None:
            ybar, T, Ci = cast(ybar), cast(T), cast(Ci)
        cib = np.zeros_like(T)
        tbar = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
        tb.append(tbar[lk, lj, li])
        cb.append(cib[lk, lj, li])
    return np.array(tb), np.array(cb)


def test_fp64_transposed_step_past_2e31_elements():
    """The FP64 transposed step on the pre-scaled coefficient at 1296^3 (element offsets
    past 2^31): Tbar and dL/dCi at samples - interior, faces, edges - against the
    oracle's transposed step on each sample's block."""
    n = N_BIG
    dev = torch.device("cuda")
    T, C = big_fields(dev)
    ybar = inputs.uniform_field_torch(SEED_YBAR_BIG, n, n, n, dev)
    ybar -= 0.5
    dt = api.stable_dt(C, 1.0)
    inv = inputs.inverse_spacing(n, n, n)
    api.scale_ci(C, 1.0, dt, inv, out=C)  # in place: Cs
    Tbar, Csbar = torch.empty_like(T), torch.zeros_like(T)
    api.adjoint(Tbar, Csbar, ybar, T, C, 1.0, dt, inv, ci_scaled=True)
    del T, C, ybar
    api.scale_ci(Csbar, 1.0, dt, inv, out=Csbar)  # dL/dCi = dt*lam*_dx^2 * dL/dCs
    got_t, got_c = sample(Tbar, PTS_BIG), sample(Csbar, PTS_BIG)
    ref_t, ref_c = adjoint_refs(adjoint_blocks(PTS_BIG, n), 1.0, dt, inv)
    assert np.max(np.abs(got_t - ref_t)) <= 1e-14
    assert np.max(np.abs(got_c - ref_c)) <= 1e-12 * np.max(np.abs(ref_c))
    assert np.count_nonzero(ref_c) >= 3  # interior samples carry a dL/dCi term
    assert api.device_error() == 0
    del Tbar, Csbar
    torch.cuda.empty_cache()


def test_fp32_transposed_step_past_2e31_elements():
    """The same on FP32 fields (the states in deviation storage), against the oracle on the
    FP32-rounded inputs."""
    n = N_BIG
    dev = torch.device("cuda")
    D = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    C32, Y = torch.empty_like(D), torch.empty_like(D)
    for k0 in range(0, n, 64):  # FP64 draws a slab at a time, rounded to FP32 like the host
        k1 = min(n, k0 + 64)
        idx = torch.arange(k0 * n * n, k1 * n * n, dtype=torch.int64, device=dev)
        D[k0:k1] = ((inputs.T_BASE + inputs.uniform_torch(SEED_T_BIG, idx)) - inputs.T_BASE).view(k1 - k0, n, n)
        C32[k0:k1] = (((inputs.uniform_torch(inputs.SEED_CI, idx) * 0.5) + 1.0) * (1.0 / inputs.C0)).view(
            k1 - k0, n, n)
        Y[k0:k1] = (inputs.uniform_torch(SEED_YBAR_BIG, idx) - 0.5).view(k1 - k0, n, n)
    dt = api.stable_dt(C32, 1.0)
    inv = inputs.inverse_spacing(n, n, n)
    Tbar, Cib = torch.empty_like(D), torch.zeros_like(D)
    api.adjoint(Tbar, Cib, Y, D, C32, 1.0, dt, inv)
    del D, C32, Y
    got_t, got_c = sample(Tbar, PTS_BIG), sample(Cib, PTS_BIG)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    blocks = [(loc, ybar, T - inputs.T_BASE, Ci) for loc, ybar, T, Ci in adjoint_blocks(PTS_BIG, n)]
    ref_t, ref_c = adjoint_refs(blocks, 1.0, dt, inv, cast=f32)
    assert np.max(np.abs(got_t - ref_t)) <= 2e-6 * np.max(np.abs(ref_t))
    assert np.max(np.abs(got_c - ref_c)) <= 2e-6 * np.max(np.abs(ref_c))
    assert np.count_nonzero(ref_c) >= 3
    assert api.device_error() == 0
    del Tbar, Cib
    torch.cuda.empty_cache()
