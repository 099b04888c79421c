"""Batched step on the TMA z-march kernel (one CTA per work item, the single-grid
step's tile body) and the batch's row pitch.

Pins: a batched problem equals its own single run bit for bit (same arithmetic,
same tile); results do not depend on the row pitch or the z-chunk length; odd
sizes (padded rows) match the FP64 oracle; the kernel choice and its refusals."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import _lib, api, tuner

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FP64_TOL = 1e-12
U32 = 2.0 ** -24


def f32(a):
    return a.astype(np.float32).astype(np.float64)


def f32_tol(nt, D0):
    """The FP32 bound of the parity tests: 13 roundings of max|D| per step."""
    return nt * 13 * U32 * float(np.max(np.abs(D0)))


def fields(shape, q, dtype, seed0=3000):
    """Workload-shaped fields on a grid with one spacing d = 1/(max n - 1) on every
    axis (the FP64 z-march takes equal spacings) and Fig. 1's dt."""
    nx, ny, nz = shape
    T0, Ci, lam, _, _ = problem(nx, ny, nz, seed=seed0 + q)
    d = 1.0 / (max(shape) - 1)
    dt = d * d / lam / Ci.max() / 6.1
    if dtype == torch.float32:
        T0, Ci = f32(T0 - 1.7), f32(Ci)
    return T0, Ci, lam, dt, (1.0 / d,) * 3


def make_batch_problems(shapes, dtype, pitched, seed0=3000):
    probs, host = [], []
    for q, shape in enumerate(shapes):
        T0, Ci, lam, dt, inv = fields(shape, q, dtype, seed0)
        T, C = to_dev(T0, dtype), to_dev(Ci, dtype)
        if pitched:
            T, C = api.pitched_copy(T), api.pitched_copy(C)
        T2 = api.pitched_copy(T) if pitched else T.clone()
        probs.append(dict(T=T, T2=T2, Ci=C, lam=lam, dt=dt, inv_spacing=inv))
        host.append((T0, Ci, lam, dt, inv))
    return probs, host


def single_run(T0, Ci, lam, dt, inv, nt, dtype, ci_scaled=False):
    T = to_dev(T0, dtype)
    C = to_dev(Ci, dtype)
    if ci_scaled:
        C = api.scale_ci(C, lam, dt, inv)
    return api.run(T, T.clone(), C, lam, dt, inv, nt, graph=False, ci_scaled=ci_scaled)


# shapes whose single runs take the TMA step kernel (rows of a multiple of 16 bytes)
EVEN64 = [(32, 32, 32), (34, 21, 9), (64, 64, 64), (66, 17, 30), (130, 40, 12), (4, 3, 3)]
EVEN32 = [(32, 32, 32), (36, 21, 9), (128, 16, 12), (132, 40, 12), (4, 3, 3), (260, 9, 5)]


@pytest.mark.parametrize("dtype,shapes,prescale", [(torch.float64, EVEN64, True), (torch.float64, EVEN64, False),
                                                    (torch.float32, EVEN32, True)])
@pytest.mark.parametrize("nt", [1, 6])
def test_zmarch_batch_equals_single_runs(dtype, shapes, prescale, nt):
    """FP64 problems on Ci as given are stepped on the batch's own pre-scaled copy by
    default (equal to the pre-scaled single run), else on Ci as given (equal to that
    single run); FP32 is never pre-scaled."""
    probs, host = make_batch_problems(shapes, dtype, pitched=False)
    b = api.Batch(probs, kernel="zmarch", prescale=prescale)
    assert b.kernel == "zmarch"
    assert b.prescaled == (prescale and dtype == torch.float64)
    b.run(nt, graph=False)
    for q, h in enumerate(host):
        ref = single_run(*h, nt, dtype, ci_scaled=b.prescaled)
        assert torch.equal(b.result(q, nt), ref), q
    assert api.device_error() == 0


def test_prescaled_batch_keeps_the_given_ci_and_pitch():
    """The batch's own Cs copies leave the caller's Ci untouched; padded rows work."""
    probs, host = make_batch_problems([(33, 33, 33), (47, 31, 20)], torch.float64, pitched=True)
    before = [p["Ci"].clone() for p in probs]
    b = api.Batch(probs)
    assert b.prescaled and b.kernel == "zmarch"
    b.run(3, graph=False)
    for p, c in zip(probs, before):
        assert torch.equal(p["Ci"], c)
    for q, h in enumerate(host):
        ref = single_run(*h, 3, torch.float64, ci_scaled=True)
        assert torch.equal(b.result(q, 3).contiguous(), ref), q


ODD = [(3, 3, 3), (5, 7, 6), (17, 17, 17), (33, 33, 33), (47, 31, 20), (61, 9, 70), (97, 40, 13),
       (131, 5, 8), (160, 12, 10)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_zmarch_batch_padded_rows_match_oracle(dtype):
    nt = 5
    probs, host = make_batch_problems(ODD, dtype, pitched=True)
    b = api.Batch(probs)  # every problem qualifies once its rows are padded
    assert b.kernel == "zmarch"
    b.run(nt, graph=True)
    for q, (T0, Ci, lam, dt, inv) in enumerate(host):
        ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
        got = to_host(b.result(q, nt))
        if dtype == torch.float64:
            assert rel_linf(got, ref) <= FP64_TOL, q
        else:
            assert np.max(np.abs(got - ref)) <= f32_tol(nt, T0) + 1e-30, q
    assert api.device_error() == 0
    api.clear_graph_cache()


@pytest.mark.parametrize("dtype,shapes", [(torch.float64, EVEN64), (torch.float32, EVEN32)])
def test_zmarch_batch_pitch_and_chunk_invariance(dtype, shapes):
    nt = 4
    out = []
    for pitched, tile in ((False, (0, 0, 0)), (True, (0, 0, 0)), (True, (0, 0, 1)), (True, (0, 0, 3)),
                          (True, (0, 0, 64))):
        probs, _ = make_batch_problems(shapes, dtype, pitched)
        b = api.Batch(probs, tile=tile, kernel="zmarch")
        b.run(nt, graph=False)
        out.append([b.result(q, nt).contiguous() for q in range(len(shapes))])
    for other in out[1:]:
        for a, c in zip(out[0], other):
            assert torch.equal(a, c)


def test_zmarch_batch_ci_scaled_equals_single_runs():
    nt = 5
    shapes = EVEN64 + [(33, 33, 33), (47, 31, 20)]
    probs, host = [], []
    for q, shape in enumerate(shapes):
        T0, Ci, lam, dt, inv = fields(shape, q, torch.float64)
        T = api.pitched_copy(to_dev(T0))
        Cs = api.pitched_copy(api.scale_ci(to_dev(Ci), lam, dt, inv))
        probs.append(dict(T=T, T2=api.pitched_copy(T), Ci=Cs, lam=lam, dt=dt, inv_spacing=inv))
        host.append((T0, Ci, lam, dt, inv))
    b = api.Batch(probs, ci_scaled=True)
    assert b.kernel == "zmarch"
    b.run(nt, graph=True)
    for q, h in enumerate(host):
        ref = single_run(*h, nt, torch.float64, ci_scaled=True)
        assert torch.equal(b.result(q, nt).contiguous(), ref), q
    api.clear_graph_cache()


def test_kernel_choice_and_refusals():
    probs, _ = make_batch_problems([(33, 33, 33), (32, 32, 32)], torch.float64, pitched=False)
    assert api.Batch(probs).kernel == "column"  # odd rows are not 16-byte aligned
    with pytest.raises(_lib.PsError) as e:
        api.Batch(probs, kernel="zmarch")
    assert e.value.status == _lib.PS_ERR_UNSUPPORTED
    with pytest.raises(_lib.PsError):
        api.Batch(probs, kernel="column", ci_scaled=True)
    p32, _ = make_batch_problems([(32, 32, 32)], torch.float32, pitched=True)
    with pytest.raises(_lib.PsError):
        api.Batch(p32, ci_scaled=True)
    # unequal FP64 spacings: the z-march path takes only equal spacings
    T0, Ci, lam, dt, inv = problem(32, 16, 8)
    assert inv[0] != inv[1]
    T = to_dev(T0)
    aniso = [dict(T=T, T2=T.clone(), Ci=to_dev(Ci), lam=lam, dt=dt, inv_spacing=inv)]
    assert api.Batch(aniso).kernel == "column"
    with pytest.raises(_lib.PsError):
        api.Batch(aniso, kernel="zmarch")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_column_kernel_with_pitch_matches_oracle(dtype):
    nt = 4
    probs, host = make_batch_problems(ODD[:6], dtype, pitched=True)
    b = api.Batch(probs, kernel="column")
    assert b.kernel == "column"
    b.run(nt, graph=False)
    for q, (T0, Ci, lam, dt, inv) in enumerate(host):
        ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
        got = to_host(b.result(q, nt))
        if dtype == torch.float64:
            assert rel_linf(got, ref) <= FP64_TOL, q
        else:
            assert np.max(np.abs(got - ref)) <= f32_tol(nt, T0) + 1e-30, q


def test_column_entry_point_refuses_zmarch_table():
    """The column-march step call given a z-march table leaves the fields alone and
    sets bit 1 of the device flags."""
    probs, _ = make_batch_problems([(32, 32, 32)], torch.float64, pitched=True)
    b = api.Batch(probs)
    assert b.kernel == "zmarch"
    before = probs[0]["T2"].clone()
    lib = _lib.load()
    _lib.check(lib.ps_diffusion3d_batch_step(b.table.data_ptr(), 0, _lib.PS_F64,
                                             torch.cuda.current_stream().cuda_stream))
    assert api.device_error(clear=True) == 2
    assert torch.equal(probs[0]["T2"], before)
    assert api.device_error() == 0


def test_tuned_zmarch_batch(tmp_path, monkeypatch):
    import json
    monkeypatch.setenv("PS_TUNER_CACHE", str(tmp_path / "tuner.json"))
    shapes = [(34, 34, 34), (50, 50, 50), (90, 90, 90), (131, 131, 131)]
    nt = 3
    probs, host = make_batch_problems(shapes, torch.float64, pitched=True)
    best = tuner.tune(probs, reps=2)
    cache = json.load(open(tmp_path / "tuner.json"))
    assert all("|zmarch" in k for k in cache)  # "zmarch-scaled": FP64 is stepped on its own Cs
    assert all(tuple(v) in tuner.ZMARCH_CANDIDATES for v in cache.values())
    b = tuner.tuned_batch(probs)  # timing steps the fields: reset them afterwards
    for p, (T0, *_rest) in zip(probs, host):
        p["T"].copy_(to_dev(T0))
        p["T2"].copy_(p["T"])
    assert b.kernel == "zmarch" and len(best) >= 1
    b.run(nt, graph=False)
    for q, (T0, Ci, lam, dt, inv) in enumerate(host):
        assert rel_linf(to_host(b.result(q, nt)), oracle.run(T0, Ci, lam, dt, *inv, nt)) <= FP64_TOL


ZITEM = [("prob", "<i4"), ("i0", "<i4"), ("j0", "<i4"), ("k0", "<i4"), ("ni", "<i2"), ("nj", "<i2"),
         ("nk", "<i2"), ("kind", "<i2")]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_zmarch_table_covers_every_interior_node_once(dtype):
    """Wide tiles (one warp per row, 8 rows) from the origin, a narrow last tile (half
    a warp per row, 16 rows) where at most half a wide tile of columns is left; every
    interior node in exactly one item; problems largest first, each one's items
    together."""
    sizes = [3, 4, 34, 35, 65, 66, 67, 97, 98, 129, 130, 131, 160]
    shapes = [(n, (n % 7) + 3, (n % 5) + 3) for n in sizes]
    probs, _ = make_batch_problems(shapes, dtype, pitched=True)
    b = api.Batch(probs, tile=(0, 0, 2))
    assert b.kernel == "zmarch"
    raw = bytes(b.host)
    ioff = int(np.frombuffer(raw[40:48], dtype=np.int64)[0])
    items = np.frombuffer(raw[ioff:ioff + 24 * b.nitems], dtype=np.dtype(ZITEM))
    wide = 64 if dtype == torch.float64 else 128
    covered = {q: np.zeros(s[::-1], dtype=np.int32) for q, s in enumerate(shapes)}
    seen = []
    for it in items:
        q, x0, y0, k0, nk, kind = (int(it[f]) for f in ("prob", "i0", "j0", "k0", "nk", "kind"))
        nx, ny, nz = shapes[q]
        bx, by = (wide, 8) if kind == 0 else (wide // 2, 16)
        assert x0 % wide == 0 and 1 <= k0 and k0 + nk <= nz - 1 and 1 <= nk <= 2
        if kind == 1:
            assert nx - 1 - x0 <= wide // 2
        covered[q][k0:k0 + nk, max(y0, 1):min(y0 + by, ny - 1), max(x0, 1):min(x0 + bx, nx - 1)] += 1
        if not seen or seen[-1] != q:
            seen.append(q)
    for q, (nx, ny, nz) in enumerate(shapes):
        c = covered[q]
        assert c[1:-1, 1:-1, 1:-1].min() == 1 and c.max() == 1 and c.sum() == (nx - 2) * (ny - 2) * (nz - 2)
    assert sorted(seen) == list(range(len(shapes)))  # each problem's items are contiguous
    vols = [np.prod(shapes[q]) for q in seen]
    assert vols == sorted(vols, reverse=True)


# ------------------------------------------------------------ fused step pairs
def pair_problems(dtype, shapes, seed0=4000):
    """Pitched problems; FP64 ones on the pre-scaled coefficient (pairs need it)."""
    probs, host = make_batch_problems(shapes, dtype, pitched=True, seed0=seed0)
    if dtype == torch.float64:
        for p in probs:
            p["Ci"] = api.pitched_copy(api.scale_ci(p["Ci"].contiguous(), p["lam"], p["dt"], p["inv_spacing"]))
    return probs, host


PAIR_SHAPES = [(3, 3, 3), (17, 17, 17), (33, 33, 33), (64, 20, 9), (67, 70, 12), (130, 9, 33),
               (161, 12, 10)]


def reset(probs, host, dtype):
    for p, (T0, *_r) in zip(probs, host):
        p["T"].copy_(to_dev(T0, dtype))
        p["T2"].copy_(p["T"])


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_pairs_equal_single_steps(dtype, graph):
    """Fused pairs give bit for bit the single steps, whatever the pair count's
    parity (an odd count runs one pair as two steps) and the z-chunk length."""
    scaled = dtype == torch.float64
    probs, host = pair_problems(dtype, PAIR_SHAPES)
    one = api.Batch(probs, ci_scaled=scaled)
    two = api.Batch(probs, tile=(0, 0, 5), ci_scaled=scaled, temporal2=True)
    for nt in (1, 2, 3, 4, 5, 6, 7):
        reset(probs, host, dtype)
        one.run(nt, graph=graph)
        ref = [one.result(q, nt).clone() for q in range(len(probs))]
        reset(probs, host, dtype)
        two.run(nt, graph=graph)
        for q in range(len(probs)):
            assert torch.equal(two.result(q, nt), ref[q]), (nt, q)
    assert api.device_error() == 0
    api.clear_graph_cache()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_step2_is_two_steps(dtype):
    scaled = dtype == torch.float64
    probs, host = pair_problems(dtype, PAIR_SHAPES[:4])
    b = api.Batch(probs, ci_scaled=scaled, temporal2=True)
    b.step(0)
    b.step(1)
    ref = [p["T"].clone() for p in probs]
    reset(probs, host, dtype)
    b.step2(0)  # T -> T2 after two steps
    for q, p in enumerate(probs):
        assert torch.equal(p["T2"], ref[q]), q


def test_batch_pairs_refusals():
    p64, _ = make_batch_problems([(32, 32, 32)], torch.float64, pitched=True)
    with pytest.raises(_lib.PsError):  # FP64 pairs run on the pre-scaled coefficient only
        api.Batch(p64, temporal2=True, prescale=False)
    assert api.Batch(p64, temporal2=True).prescaled  # the batch's own Cs serves them
    p32, _ = make_batch_problems([(32, 32, 32)], torch.float32, pitched=True)
    with pytest.raises(_lib.PsError):
        api.Batch(p32, kernel="column", temporal2=True)
    b = api.Batch(p32)
    lib = _lib.load()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.ps_diffusion3d_batch_run_ex(b.table.data_ptr(), b.host, 4, _lib.PS_RUN_TEMPORAL2, s) == \
        _lib.PS_ERR_ARG
    assert lib.ps_diffusion3d_batch_step2_ex(b.table.data_ptr(), b.host, 0, s) == _lib.PS_ERR_ARG


def test_tuned_depth_is_cached_and_correct(tmp_path, monkeypatch):
    import json
    monkeypatch.setenv("PS_TUNER_CACHE", str(tmp_path / "tuner.json"))
    nt = 6
    probs, host = pair_problems(torch.float32, [(40, 40, 40), (90, 90, 90), (131, 131, 131)])
    depth = tuner.tune_depth(probs, reps=2)
    assert depth in (1, 2)
    cache = json.load(open(tmp_path / "tuner.json"))
    assert [v for k, v in cache.items() if "depth" in k] == [[depth]]
    reset(probs, host, torch.float32)
    b = tuner.tuned_batch(probs, reps=2)
    assert b.temporal2 == (depth == 2)
    b.run(nt, graph=False)
    for q, (T0, Ci, lam, dt, inv) in enumerate(host):
        ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
        assert np.max(np.abs(to_host(b.result(q, nt)) - ref)) <= f32_tol(nt, T0) + 1e-30
