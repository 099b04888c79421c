"""Gradients of L = 1/2||T(nt) - T_obs||^2 through the CUDA path (hand-written
transposed step + sqrt(nt) checkpointing) against the FP64 oracle's gradient
and central finite differences."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import api, inputs
from paper_2211_15634_gb300 import autograd as ag

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def inverse_problem(nx, ny, nz, nt):
    """Config of the inverse problem on a small grid: T_obs from the smooth true Ci,
    the loss evaluated at Ci = 1/c0 plus a small seeded perturbation."""
    lam = 1.0
    T0 = inputs.t0_gaussian(nx, ny, nz)
    Ci_true = inputs.ci_smooth(nx, ny, nz)
    Ci = inputs.ci_constant(nx, ny, nz) + 0.02 * inputs.random_field((nz, ny, nx), 8)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / (1.5 / inputs.C0) / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    Tobs = oracle.run(T0, Ci_true, lam, dt, *inv, nt)
    return T0, Ci, Tobs, lam, dt, inv


@pytest.mark.parametrize("shape,nt", [((24, 20, 28), 12), ((33, 17, 21), 9), ((68, 40, 30), 16)])
def test_gradient_matches_oracle_fp64(shape, nt):
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(*shape, nt)
    L_ref, dT0_ref, dCi_ref = oracle.gradient(T0, Ci, Tobs, lam, dt, *inv, nt)
    L, dT0, dCi = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt)
    assert abs(float(L) - L_ref) <= 1e-12 * L_ref
    assert rel_linf(to_host(dT0), dT0_ref) <= 1e-10
    assert rel_linf(to_host(dCi), dCi_ref) <= 1e-10


def test_gradient_fp32_error_reported_bound():
    """FP32 path (deviation storage): the gradient stays within 1e-3 relative of
    the FP64 oracle's (FP32 rounding accumulated over nt forward and nt adjoint steps)."""
    nx, ny, nz, nt = 36, 20, 24, 10
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    L_ref, dT0_ref, dCi_ref = oracle.gradient(T0, Ci, Tobs, lam, dt, *inv, nt)
    D0 = api.to_deviation(to_dev(T0), 1.7)
    Dobs = api.to_deviation(to_dev(Tobs), 1.7)
    C32 = api.to_f32(to_dev(Ci))
    L, dT0, dCi = ag.loss_and_grad(D0, C32, Dobs, lam, dt, inv, nt)
    assert abs(float(L) - L_ref) <= 1e-4 * L_ref
    assert rel_linf(to_host(dT0), dT0_ref) <= 1e-3
    assert rel_linf(to_host(dCi), dCi_ref) <= 1e-3


def test_autograd_function_matches_loss_and_grad():
    nx, ny, nz, nt = 28, 18, 20, 11
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    T0d = to_dev(T0).requires_grad_(True)
    Cid = to_dev(Ci).requires_grad_(True)
    out = ag.Diffusion3DFn.apply(T0d, Cid, lam, dt, inv, nt)
    L = 0.5 * ((out - to_dev(Tobs)) ** 2).sum()
    gT0, gCi = torch.autograd.grad(L, (T0d, Cid))
    L2, dT0, dCi = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt)
    assert rel_linf(to_host(gT0), to_host(dT0)) <= 1e-13
    assert rel_linf(to_host(gCi), to_host(dCi)) <= 1e-13


@pytest.mark.parametrize("every", [1, 4])
def test_kept_output_does_not_hold_the_state_block(every):
    """T(nt) from Diffusion3DFn owns its storage: after backward, keeping the output
    holds one field, not the block of checkpoints it was stepped in."""
    nx, ny, nz, nt = 40, 32, 36, 16
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    T0d = to_dev(T0).requires_grad_(True)
    Cid = to_dev(Ci).requires_grad_(True)
    Tobsd = to_dev(Tobs)
    field = T0.nbytes
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    out = ag.Diffusion3DFn.apply(T0d, Cid, lam, dt, inv, nt, every)
    L = 0.5 * ((out - Tobsd) ** 2).sum()
    gT0, gCi = torch.autograd.grad(L, (T0d, Cid))
    del L, gT0, gCi
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - before
    assert out.untyped_storage().nbytes() == field
    assert held <= field + 4096, f"{held} bytes held with the output, one field is {field}"
    del out
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - before <= 4096


@pytest.mark.parametrize("every", [1, 2, 5, 13])
def test_checkpoint_interval_does_not_change_gradient(every):
    """Recomputed states are bit-identical to the forward ones, so any interval
    gives the same gradient bit for bit."""
    nx, ny, nz, nt = 24, 14, 18, 13
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    base = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt, every=nt)
    got = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt, every=every)
    for a, b in zip(base, got):
        assert torch.equal(a, b)


@pytest.mark.parametrize("every", [2, 3, 4, 6])
def test_one_stream_sweep_gives_the_same_gradient(every):
    """The sweep without the side stream (recompute, then transposed steps, on one
    stream; the kept last two segments, then each recompute in the block of the segment
    swept before it): bit for bit the gradient of the one-segment run."""
    nx, ny, nz, nt = 24, 14, 18, 13
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    base = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt, every=nt)
    T0d, Cid, Tobsd = to_dev(T0), to_dev(Ci), to_dev(Tobs)
    coef = ag.coefficient(Cid, lam, dt, inv)
    out, ckpts, kept = ag.forward_checkpointed(T0d, Cid, lam, dt, inv, nt, every, coef)
    assert len(ckpts) == (nt - 1) // every + 1 and sorted(kept) == [len(ckpts) - 2, len(ckpts) - 1]
    resid = torch.empty_like(out)
    L = api.half_sq_dist(out, Tobsd, residual=resid)
    dT0, dCi = ag.backward_checkpointed(resid, Cid, lam, dt, inv, nt, every, ckpts, coef, overlap=False,
                                        kept=kept)
    for a, b in zip(base, (L, dT0, dCi)):
        assert torch.equal(a, b)


def test_gradient_central_differences_16():
    """Directional derivatives of the GPU loss against central differences of GPU
    forward runs on 16^3 (relative 1e-6)."""
    n, nt = 16, 20
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(n, n, n, nt)
    T0d, Cid, Tobsd = to_dev(T0), to_dev(Ci), to_dev(Tobs)
    L, dT0, dCi = ag.loss_and_grad(T0d, Cid, Tobsd, lam, dt, inv, nt)

    def loss(t0, ci):
        a, b = t0.clone(), t0.clone()
        out = api.run(a, b, ci, lam, dt, inv, nt)
        return float(api.half_sq_dist(out, Tobsd))

    v = to_dev(inputs.random_field((n, n, n), 9))
    h = 1e-4
    fd = (loss(T0d, Cid + h * v) - loss(T0d, Cid - h * v)) / (2 * h)
    ad = float(api.dot(dCi, v))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    w = to_dev(inputs.random_field((n, n, n), 10))
    h = 1e-3
    fd = (loss(T0d + h * w, Cid) - loss(T0d - h * w, Cid)) / (2 * h)
    ad = float(api.dot(dT0, w))
    assert abs(fd - ad) <= 1e-6 * abs(ad)


@pytest.mark.parametrize("kchunk", ["0", "3", "40"])
def test_adjoint_fixed_point_scale_growth(launch_override, kchunk):
    """ybar growing by 10^4 along z (with sign changes and exact zeros) makes the
    FP64 adjoint's per-CTA fixed-point scale grow in the middle of its z-march,
    so tiles already stored must be rescaled; results still match the oracle."""
    launch_override(adj_kchunk=kchunk)
    nx, ny, nz = 68, 21, 40
    T = 1.7 + inputs.random_field((nz, ny, nx), 3, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    lam = 1.0
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci.max() / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    ybar = inputs.random_field(T.shape, 5) * (10.0 ** (np.arange(nz) / 10.0))[:, None, None]
    ybar[:, ::4, ::3] = 0.0
    cib = inputs.random_field(T.shape, 6)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    Tbar = torch.empty(T.shape, dtype=torch.float64, device="cuda")
    C = to_dev(inputs.random_field(T.shape, 6))
    api.adjoint(Tbar, C, to_dev(ybar), to_dev(T), to_dev(Ci), lam, dt, inv)
    # error relative to each plane's own scale (planes differ by up to 10^4)
    got = to_host(Tbar)
    for k in range(nz):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-13 * np.max(np.abs(ref[k])), k
    assert np.max(np.abs(to_host(C) - cib)) <= 1e-13 * np.max(np.abs(cib))


@pytest.mark.parametrize("kchunk", ["1", "2", "5"])
def test_adjoint_short_z_chunks(launch_override, kchunk):
    launch_override(adj_kchunk=kchunk)
    nx, ny, nz = 132, 19, 13
    T = 1.7 + inputs.random_field((nz, ny, nx), 3, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    lam = 1.0
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci.max() / 6.1
    inv = inputs.inverse_spacing(nx, ny, nz)
    ybar = inputs.random_field(T.shape, 5)
    cib = np.zeros_like(T)
    ref = oracle.adjoint_step(ybar, T, Ci, cib, lam, dt, *inv)
    for dtype, tol in ((torch.float64, 1e-14), (torch.float32, 1e-5)):
        Tbar = torch.empty(T.shape, dtype=dtype, device="cuda")
        C = torch.zeros(T.shape, dtype=dtype, device="cuda")
        api.adjoint(Tbar, C, to_dev(ybar, dtype), to_dev(T, dtype), to_dev(Ci, dtype), lam, dt, inv)
        assert rel_linf(to_host(Tbar), ref) <= tol
        assert np.max(np.abs(to_host(C) - cib)) <= tol * np.max(np.abs(cib))
    assert api.device_error() == 0


def test_default_interval_keeps_every_state_when_it_fits():
    """every=None: a small grid's nt states fit, so every state is kept (interval 1);
    the gradient equals the sqrt(nt)-checkpoint one bit for bit."""
    nx, ny, nz, nt = 24, 14, 18, 13
    T0, Ci, Tobs, lam, dt, inv = inverse_problem(nx, ny, nz, nt)
    assert ag.auto_every(to_dev(T0), nt) == 1
    auto = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt)
    sq = ag.loss_and_grad(to_dev(T0), to_dev(Ci), to_dev(Tobs), lam, dt, inv, nt,
                          every=ag.default_every(nt))
    for a, b in zip(auto, sq):
        assert torch.equal(a, b)
