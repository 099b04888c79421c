"""Differentiable time loop: T(nt) = M(Ci)^nt T0 with hand-written adjoint.

``Diffusion3DFn.apply(T0, Ci, lam, dt, inv_spacing, nt, every)`` runs the
Fig. 1 time loop forward, keeping a checkpoint of the state every ``every``
steps.  By default (``every=None``) every state is kept when the nt fields fit
in the device's free memory with a margin (no recompute: the reverse sweep
reads each state once), else every ``ceil(sqrt(nt))`` steps.  ``backward`` walks the
segments in reverse: it recomputes the states of one segment from its
checkpoint with the forward kernel (the last two segments' states are kept from the
forward pass, which computes them anyway; on FP32 grids the forward's loops that
keep every state run fused step pairs that write both states), then applies the transposed step
(``ps_diffusion3d_adjoint``) from the segment's last step to its first,
accumulating dL/dCi; the next segment's recompute runs on a side stream meanwhile.
dt is held constant (not differentiated through maximum(Ci)).  Memory: about
``nt/every + 2*every + 2`` fields.

On FP64 grids with equal spacings every kernel runs on the pre-scaled
coefficient Cs = dt*lam*_dx^2*Ci (one FP64 multiply-add per node forward);
the sweep then accumulates dL/dCs and returns dL/dCi = dt*lam*_dx^2 * dL/dCs.
With ``pairs=True`` (FP32 grids) the reverse sweep takes the transposed steps
two at a time (``api.adjoint2``: one pass over HBM per pair, bit for bit two
single steps; measured no faster than single steps on GB300, so off by default).
"""
from __future__ import annotations

import math

import torch

from . import api


def default_every(nt: int) -> int:
    """The sqrt(nt) checkpoint interval."""
    return max(1, int(math.ceil(math.sqrt(nt))))


# fields the sweep holds besides the states: the coefficient (and Cs), the residual,
# ybar / Tbar, dL/dCi (or dL/dCs) and the two gradients returned
WORK_FIELDS = 8


def choose_every(nt: int, field_bytes: int, free_bytes: int, margin: float = 0.8) -> int:
    """1 (every state kept) when nt state fields and the sweep's working fields fit in
    ``margin`` of ``free_bytes``; else the sqrt(nt) interval."""
    if (nt + WORK_FIELDS) * field_bytes <= margin * free_bytes:
        return 1
    return default_every(nt)


def auto_every(T0: torch.Tensor, nt: int) -> int:
    """Checkpoint interval for T0's device: free memory as the driver reports it plus
    what the caching allocator holds unused."""
    if not T0.is_cuda:
        return default_every(nt)
    free, _ = torch.cuda.mem_get_info(T0.device)
    free += torch.cuda.memory_reserved(T0.device) - torch.cuda.memory_allocated(T0.device)
    return choose_every(nt, T0.numel() * T0.element_size(), free)


def coefficient(Ci, lam, dt, inv):
    """(field the kernels read, pre-scaled?): Cs = dt*lam*_dx^2*Ci on FP64 grids
    with equal spacings, else Ci itself."""
    if Ci.dtype == torch.float64 and inv[0] == inv[1] == inv[2]:
        return api.scale_ci(Ci, lam, dt, inv), True
    return Ci, False


def state_pairs_default(T0) -> bool:
    """Whether the forward pass's state-keeping loops run fused step pairs that write both
    states (``api.run_states(temporal2=True)``: FP32 only; bit for bit the same states).
    Measured at 256^3, nt = 200: 200 states in 5.74 against 6.71 ms, the gradient with every
    state kept 18.52 against 19.52 ms.  The reverse sweep's recomputes stay single steps by
    default: there they run beside the transposed steps, and in pairs the sqrt(nt)
    gradient measured slower (22.00 against 21.80 ms)."""
    return T0.dtype == torch.float32


def forward_checkpointed(T0, Ci, lam, dt, inv, nt, every, coef=None, graph=True, state_pairs=None):
    """Run nt steps; return (final state, [checkpoint at step 0, every, 2*every, ...], kept).

    ``kept`` maps each of the last two segments to a :class:`api.StateBlock` of ``every``
    grids holding its states (after its steps 1, 2, ...) - the forward computes them
    anyway, and the reverse sweep needs two segment buffers, so it takes these two
    segments without recomputing them (None when every state is kept).  ``coef`` =
    :func:`coefficient` (computed here when None).  ``graph``: replay the state-keeping
    loops from the library's graph cache (keyed by the buffers, which the caching
    allocator hands back unchanged in a loop of gradients).  ``state_pairs``: the loops
    run fused step pairs (default :func:`state_pairs_default`)."""
    C, scaled = coefficient(Ci, lam, dt, inv) if coef is None else coef
    pairs = state_pairs_default(T0) if state_pairs is None else bool(state_pairs)
    if nt == 0:
        return T0.clone(), [T0], None
    if every == 1:
        # every state in one block; the steps write straight into it (one library call)
        block = api.StateBlock(T0, nt, boundary=False)  # run_states sets the boundaries
        cur = api.run_states(T0, block, 1, C, lam, dt, inv, nt, ci_scaled=scaled, graph=graph, temporal2=pairs)
        return cur, [T0] + block.grids[:nt - 1], None
    nseg = (nt - 1) // every + 1
    first_kept = max(0, nseg - 2)
    t_keep = first_kept * every  # checkpoint step where the kept segments start
    ckpts = [T0]
    if t_keep > 0:
        # checkpoints (the state after every `every`-th step) and two work grids in one block
        block = api.StateBlock(T0, t_keep // every + 2, boundary=False)
        api.run_states(T0, block, every, C, lam, dt, inv, t_keep, ci_scaled=scaled, graph=graph, temporal2=pairs)
        ckpts += block.grids[:t_keep // every]
    kept = {}
    cur = ckpts[-1]
    for s in range(first_kept, nseg):
        t0, t1 = s * every, min(s * every + every, nt)
        kept[s] = api.StateBlock(T0, every, boundary=False)
        cur = api.run_states(cur, kept[s], 1, C, lam, dt, inv, t1 - t0, ci_scaled=scaled, graph=graph,
                             temporal2=pairs)
        if s + 1 < nseg:
            ckpts.append(cur)  # the checkpoint at step t1
    return cur, ckpts, kept


def backward_checkpointed(ybar_nt, Ci, lam, dt, inv, nt, every, ckpts, coef=None, pairs=None,
                          overlap=None, graph=True, kept=None, state_pairs=None):
    """Reverse sweep; returns (dL/dT0, dL/dCi).  ``pairs``: take the transposed
    steps two per launch where ``api.adjoint2`` applies (default off).  ``overlap``
    (default on for CUDA tensors when a segment is recomputed): recompute segment s-1's
    states on a side stream while segment s's transposed steps run, into a second
    segment buffer (one more segment of memory); the kernels and their order on every
    buffer are unchanged, so the gradient is bit for bit the one-stream sweep's.
    ``graph``: the segments' recomputes are replayed from the graph cache, as in
    :func:`forward_checkpointed`.  ``kept``: segments whose states the forward kept
    (:func:`forward_checkpointed`); they are not recomputed, and their blocks then serve
    as the recomputes' buffers.  ``state_pairs``: the recomputes run fused step pairs, as
    in :func:`forward_checkpointed` (default off, see :func:`state_pairs_default`)."""
    C, scaled = coefficient(Ci, lam, dt, inv) if coef is None else coef
    spairs = bool(state_pairs)
    pairs = bool(pairs) and not scaled and api.adjoint2_supported(ybar_nt)
    ybar = ybar_nt.contiguous().clone()
    tbar = torch.empty_like(ybar)
    cibar = torch.zeros_like(Ci)  # dL/dCs when scaled
    nseg = len(ckpts)
    seg_len = max(0, min(every, nt) - 1)  # recomputed states per segment
    seg_buf = dict(kept) if kept else {}  # segment -> block holding its states
    if overlap is None:
        overlap = ybar.is_cuda and nseg > 1 and seg_len > 0 and nseg > len(seg_buf)
    # the recompute of segment s writes into the block of segment s + nbuf, whose sweep is
    # done (s + 2 beside the sweep of s + 1 on the side stream; s + 1 on one stream)
    nbuf = 2 if overlap else 1
    main = torch.cuda.current_stream(ybar.device) if overlap else None
    side = torch.cuda.Stream(ybar.device) if overlap else None
    ready, swept = {}, {}  # recompute of segment s done; sweep of segment s done

    def recompute(s):
        t0 = s * every
        t1 = min(t0 + every, nt)
        if t1 - t0 <= 1 or s in seg_buf:
            return
        owner = s + nbuf
        blk = seg_buf.pop(owner, None)
        if blk is None:
            blk = api.StateBlock(ckpts[0], seg_len, boundary=False)  # run_states sets the boundaries
        seg_buf[s] = blk
        if not overlap:
            api.run_states(ckpts[s], blk, 1, C, lam, dt, inv, t1 - t0 - 1, ci_scaled=scaled, graph=graph,
                           temporal2=spairs)
            return
        with torch.cuda.stream(side):
            side.wait_stream(main)  # the checkpoints and Cs are final
            if owner in swept:
                side.wait_event(swept[owner])  # the sweep no longer reads this block
            api.run_states(ckpts[s], blk, 1, C, lam, dt, inv, t1 - t0 - 1, ci_scaled=scaled, graph=graph,
                           temporal2=spairs)
            ready[s] = torch.cuda.Event()
            ready[s].record(side)

    try:
        if overlap:
            recompute(nseg - 1)
        for s in range(nseg - 1, -1, -1):
            if overlap:
                if s >= 1:
                    recompute(s - 1)
                if s in ready:
                    main.wait_event(ready[s])
            else:
                recompute(s)
            t0 = s * every
            t1 = min(t0 + every, nt)
            states = [ckpts[s]] + (seg_buf[s].grids[:t1 - t0 - 1] if t1 - t0 > 1 else [])
            t = t1 - 1
            while t >= t0:
                if pairs and t - 1 >= t0:  # steps t and t-1 in one pass
                    api.adjoint2(tbar, cibar, ybar, states[t - t0], states[t - 1 - t0], C, lam, dt, inv)
                    t -= 2
                else:
                    api.adjoint(tbar, cibar, ybar, states[t - t0], C, lam, dt, inv, ci_scaled=scaled)
                    t -= 1
                ybar, tbar = tbar, ybar
            if overlap:
                swept[s] = torch.cuda.Event()
                swept[s].record(main)
    finally:
        if overlap:  # later work on the caller's stream (and frees of these buffers) after the side stream's
            main.wait_stream(side)
    if scaled:  # dL/dCi = dt*lam*_dx^2 * dL/dCs
        api.scale_ci(cibar, lam, dt, inv, out=cibar)
    return ybar, cibar


class Diffusion3DFn(torch.autograd.Function):
    """T(nt) from (T0, Ci); gradients through the hand-written adjoint kernel."""

    @staticmethod
    def forward(ctx, T0, Ci, lam, dt, inv_spacing, nt, every=None):
        T0 = T0.detach().contiguous()
        Ci = Ci.detach().contiguous()
        every = auto_every(T0, int(nt)) if every is None else int(every)
        coef = coefficient(Ci, lam, dt, tuple(inv_spacing))
        out, ckpts, kept = forward_checkpointed(T0, Ci, lam, dt, tuple(inv_spacing), int(nt), every, coef)
        # T(nt) lives in a state block: hand out a field of its own, so that a caller who
        # keeps T(nt) does not keep the block alive after backward
        out = out.clone()
        ctx.cfg = (lam, dt, tuple(inv_spacing), int(nt), every)
        ctx.ckpts = ckpts
        ctx.kept = kept
        ctx.coef = coef
        ctx.save_for_backward(Ci)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (Ci,) = ctx.saved_tensors
        lam, dt, inv, nt, every = ctx.cfg
        dT0, dCi = backward_checkpointed(grad_out, Ci, lam, dt, inv, nt, every, ctx.ckpts,
                                         ctx.coef, kept=ctx.kept)
        ctx.ckpts = None
        ctx.kept = None
        ctx.coef = None
        return dT0, dCi, None, None, None, None, None


def loss_and_grad(T0, Ci, Tobs, lam, dt, inv_spacing, nt, every=None, pairs=None, state_pairs=None):
    """L = 1/2||T(nt) - Tobs||^2 (FP64 on the GPU) and (dL/dT0, dL/dCi); ``every``
    as for :class:`Diffusion3DFn` (None: every state kept when it fits); ``pairs``
    as for :func:`backward_checkpointed`, ``state_pairs`` as for
    :func:`forward_checkpointed`."""
    every = auto_every(T0, int(nt)) if every is None else int(every)
    inv = tuple(inv_spacing)
    coef = coefficient(Ci.contiguous(), lam, dt, inv)
    out, ckpts, kept = forward_checkpointed(T0.contiguous(), Ci.contiguous(), lam, dt, inv, nt, every, coef,
                                            state_pairs=state_pairs)
    resid = torch.empty_like(out)
    L = api.half_sq_dist(out, Tobs, residual=resid)
    del out  # a grid of a kept block, which the sweep reuses
    dT0, dCi = backward_checkpointed(resid, Ci, lam, dt, inv, nt, every, ckpts, coef, pairs, kept=kept,
                                     state_pairs=state_pairs)
    return L, dT0, dCi
