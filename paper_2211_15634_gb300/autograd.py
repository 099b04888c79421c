"""Differentiable time loop: T(nt) = M(Ci)^nt T0 with hand-written adjoint.

``Diffusion3DFn.apply(T0, Ci, lam, dt, inv_spacing, nt, every)`` runs the
Fig. 1 time loop forward, keeping a checkpoint of the state every ``every``
steps (``every = ceil(sqrt(nt))`` by default).  ``backward`` walks the
segments in reverse: it recomputes the states of one segment from its
checkpoint with the forward kernel, then applies the transposed step
(``ps_diffusion3d_adjoint``) from the segment's last step to its first,
accumulating dL/dCi.  dt is held constant (not differentiated through
maximum(Ci)).  Memory: about ``nt/every + every + 2`` fields.
"""
from __future__ import annotations

import math

import torch

from . import api


def default_every(nt: int) -> int:
    return max(1, int(math.ceil(math.sqrt(nt))))


class _Pool:
    """Two work buffers plus the checkpoints, all with T0's boundary."""

    def __init__(self, T0: torch.Tensor):
        self.T0 = T0

    def fresh(self) -> torch.Tensor:
        t = torch.empty_like(self.T0)
        api.copy_boundary(t, self.T0)
        return t


def forward_checkpointed(T0, Ci, lam, dt, inv, nt, every):
    """Run nt steps; return (final state, [checkpoint at step 0, every, 2*every, ...])."""
    pool = _Pool(T0)
    ckpts = [T0]
    work = [pool.fresh(), pool.fresh()]
    cur = T0
    for t in range(nt):
        if (t + 1) % every == 0 and t + 1 < nt:
            dst = pool.fresh()  # the step writes straight into the next checkpoint
        else:
            dst = work[0] if cur is not work[0] else work[1]
        api.step(dst, cur, Ci, lam, dt, inv)
        cur = dst
        if (t + 1) % every == 0 and t + 1 < nt:
            ckpts.append(cur)
    if nt == 0:
        cur = T0.clone()
    return cur, ckpts


def backward_checkpointed(ybar_nt, Ci, lam, dt, inv, nt, every, ckpts):
    """Reverse sweep; returns (dL/dT0, dL/dCi)."""
    ybar = ybar_nt.contiguous().clone()
    tbar = torch.empty_like(ybar)
    cibar = torch.zeros_like(Ci)
    pool = _Pool(ckpts[0])
    seg_bufs = []
    nseg = len(ckpts)
    for s in range(nseg - 1, -1, -1):
        t0 = s * every
        t1 = min(t0 + every, nt)
        states = [ckpts[s]]
        for t in range(t0 + 1, t1):
            idx = t - t0 - 1
            if idx >= len(seg_bufs):
                seg_bufs.append(pool.fresh())
            api.step(seg_bufs[idx], states[-1], Ci, lam, dt, inv)
            states.append(seg_bufs[idx])
        for t in range(t1 - 1, t0 - 1, -1):
            api.adjoint(tbar, cibar, ybar, states[t - t0], Ci, lam, dt, inv)
            ybar, tbar = tbar, ybar
    return ybar, cibar


class Diffusion3DFn(torch.autograd.Function):
    """T(nt) from (T0, Ci); gradients through the hand-written adjoint kernel."""

    @staticmethod
    def forward(ctx, T0, Ci, lam, dt, inv_spacing, nt, every=None):
        T0 = T0.detach().contiguous()
        Ci = Ci.detach().contiguous()
        every = default_every(nt) if every is None else int(every)
        out, ckpts = forward_checkpointed(T0, Ci, lam, dt, tuple(inv_spacing), int(nt), every)
        ctx.cfg = (lam, dt, tuple(inv_spacing), int(nt), every)
        ctx.ckpts = ckpts
        ctx.save_for_backward(Ci)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (Ci,) = ctx.saved_tensors
        lam, dt, inv, nt, every = ctx.cfg
        dT0, dCi = backward_checkpointed(grad_out, Ci, lam, dt, inv, nt, every, ctx.ckpts)
        ctx.ckpts = None
        return dT0, dCi, None, None, None, None, None


def loss_and_grad(T0, Ci, Tobs, lam, dt, inv_spacing, nt, every=None):
    """L = 1/2||T(nt) - Tobs||^2 (FP64 on the GPU) and (dL/dT0, dL/dCi)."""
    every = default_every(nt) if every is None else int(every)
    inv = tuple(inv_spacing)
    out, ckpts = forward_checkpointed(T0.contiguous(), Ci.contiguous(), lam, dt, inv, nt, every)
    resid = torch.empty_like(out)
    L = api.half_sq_dist(out, Tobs, residual=resid)
    dT0, dCi = backward_checkpointed(resid, Ci, lam, dt, inv, nt, every, ckpts)
    return L, dT0, dCi
