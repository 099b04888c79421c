"""Python API over the C ABI (torch tensors for device memory and streams).

Fields are C-contiguous CUDA tensors of shape ``(nz, ny, nx)`` (x fastest),
``torch.float64`` for the FP64 path or ``torch.float32`` for the FP32 path
(which stores temperatures as deviations from a reference, see
:func:`to_deviation`).  Every function enqueues on the tensor device's
current torch stream and returns without synchronizing unless it returns a
Python float.  ``inv_spacing`` is ``(_dx, _dy, _dz)`` as in Fig. 1's
``step!`` arguments.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import PS_F32, PS_F64, check

_WS = {}


def _code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return PS_F64
    if t.dtype == torch.float32:
        return PS_F32
    raise TypeError(f"unsupported dtype {t.dtype} (need float32 or float64)")


def _field(t: torch.Tensor, name: str, code: Optional[int] = None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if code is not None and _code(t) != code:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {'float64' if code else 'float32'}")
    return t.data_ptr()


def _grid(t: torch.Tensor):
    if t.dim() != 3:
        raise ValueError("fields must have shape (nz, ny, nx)")
    nz, ny, nx = t.shape
    return nx, ny, nz


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def workspace(device) -> torch.Tensor:
    """Scratch buffer of the reductions for the device's current stream (allocated
    once per device and stream, 16 KB, reused): reductions running on different
    streams at the same time, e.g. in two :class:`SolvePipeline` objects, never share
    one."""
    device = torch.device(device)
    idx = device.index if device.index is not None else torch.cuda.current_device()
    key = (idx, torch.cuda.current_stream(idx).cuda_stream)
    ws = _WS.get(key)
    if ws is None:
        n = _lib.load().ps_workspace_bytes()
        ws = torch.empty(n, dtype=torch.uint8, device=f"cuda:{idx}")
        _WS[key] = ws
    return ws


def _same(a: torch.Tensor, *others: torch.Tensor):
    for o in others:
        if o.shape != a.shape or o.device != a.device:
            raise ValueError("fields must share shape and device")


def step(T2, T, Ci, lam: float, dt: float, inv_spacing: Sequence[float], *,
         ci_scaled: bool = False) -> None:
    """One step of Fig. 1 (``step!(T2, T, Ci, lam, dt, _dx, _dy, _dz)``).

    ``ci_scaled=True``: ``Ci`` is the pre-scaled field of :func:`scale_ci`
    (FP64, equal spacings) and the step needs one FP64 multiply-add per node.
    """
    code = _code(T)
    _same(T, T2, Ci)
    nx, ny, nz = _grid(T)
    lib = _lib.load()
    if ci_scaled:
        check(lib.ps_diffusion3d_step_ex(_field(T2, "T2", code), _field(T, "T", code),
                                         _field(Ci, "Ci", code), lam, dt, *inv_spacing, nx, ny, nz,
                                         code, _lib.PS_RUN_CI_SCALED, _stream(T)))
        return
    check(lib.ps_diffusion3d_step(_field(T2, "T2", code), _field(T, "T", code),
                                  _field(Ci, "Ci", code), lam, dt, *inv_spacing, nx, ny, nz, code,
                                  _stream(T)))


def scale_ci(Ci, lam: float, dt: float, inv_spacing, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """``Cs = dt*lam*_dx^2 * Ci`` (FP64) for ``step``/``run`` with ``ci_scaled=True``."""
    if out is None:
        out = torch.empty_like(Ci)
    check(_lib.load().ps_diffusion3d_scale_ci(_field(out, "Cs", PS_F64), _field(Ci, "Ci", PS_F64),
                                              lam, dt, inv_spacing[0], Ci.numel(), _stream(Ci)))
    return out


def step_compensated(T2, T, E2, E, Ci, lam: float, dt: float, inv_spacing) -> None:
    """Compensated FP32 step on the two-float state: the value of a node is T + E
    (FP32 deviation plus FP32 correction); (T2, E2) receives the step of that value
    with the addition done exactly (``ps_diffusion3d_step_comp_f32``)."""
    _same(T, T2, E2, E, Ci)
    nx, ny, nz = _grid(T)
    check(_lib.load().ps_diffusion3d_step_comp_f32(
        _field(T2, "T2", PS_F32), _field(T, "T", PS_F32), _field(E2, "E2", PS_F32),
        _field(E, "E", PS_F32), _field(Ci, "Ci", PS_F32), lam, dt, *inv_spacing, nx, ny, nz,
        _stream(T)))


def compensation_fields(D: torch.Tensor, E0: Optional[torch.Tensor] = None) -> torch.Tensor:
    """The two correction fields :func:`run` takes with ``comp=`` for a two-float state
    in (D, D2): shape ``(2, nz, ny, nx)`` float32, ``[0]`` paired with D (``E0`` or
    zeros), ``[1]`` with D2 (its boundary is set by the run)."""
    comp = torch.zeros((2,) + tuple(D.shape), dtype=torch.float32, device=D.device)
    if E0 is not None:
        comp[0].copy_(E0)
    return comp


def copy_boundary(T2, T) -> None:
    """T2's six boundary faces := T's (Fig. 1's ``T2 = copy(T)`` on the boundary)."""
    code = _code(T)
    _same(T, T2)
    nx, ny, nz = _grid(T)
    check(_lib.load().ps_diffusion3d_copy_boundary(_field(T2, "T2", code), _field(T, "T", code),
                                                   nx, ny, nz, code, _stream(T)))


class StateBlock:
    """``count`` state grids of T0's shape in one allocation, grid i starting
    ``stride`` elements after grid i-1 (a 16-byte boundary), every one holding
    T0's boundary (set by one launch; ``boundary=False`` leaves the grids unset, for
    :func:`run_states`, which sets the boundary of every grid it writes).
    ``grids[i]`` is grid i as a tensor."""

    def __init__(self, T0, count: int, boundary: bool = True):
        code = _code(T0)
        nx, ny, nz = _grid(T0)
        n = nx * ny * nz
        per16 = 16 // T0.element_size()
        self.stride = (n + per16 - 1) // per16 * per16
        self.flat = torch.empty(max(count, 1) * self.stride, dtype=T0.dtype, device=T0.device)
        if count and boundary:
            check(_lib.load().ps_diffusion3d_copy_boundary_many(
                self.flat.data_ptr(), count, self.stride, _field(T0, "T0", code), nx, ny, nz, code,
                _stream(T0)))
        self.grids = _GridViews(self.flat, self.stride, count, tuple(T0.shape))

    def ptr(self) -> int:
        return self.flat.data_ptr()


class _GridViews:
    """The grids of a :class:`StateBlock` as tensor views made on access (an index or a
    slice): a block of hundreds of grids costs no host time until its grids are used,
    so the steps that fill it are launched first."""

    def __init__(self, flat, stride: int, count: int, shape):
        self.flat, self.stride, self.count, self.shape = flat, stride, count, shape
        self.n = shape[0] * shape[1] * shape[2]

    def __len__(self) -> int:
        return self.count

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(self.count))]
        if i < 0:
            i += self.count
        if not 0 <= i < self.count:
            raise IndexError("state grid index out of range")
        return self.flat[i * self.stride:i * self.stride + self.n].view(self.shape)


def state_block(T0, count: int):
    """The ``count`` grids of a :class:`StateBlock` (a sequence of tensors, each made on
    access)."""
    return StateBlock(T0, count).grids


def run_states(T0, block: "StateBlock", every: int, Ci, lam: float, dt: float, inv_spacing, nt: int,
               *, ci_scaled: bool = False, graph: bool = False, temporal2: bool = False) -> torch.Tensor:
    """nt steps from T0 keeping the state after step t in grid t/every - 1 of
    ``block`` when every divides t (else in its two work grids after those);
    returns the tensor holding T(nt).  The boundary of every grid it writes is set to
    T0's (by the steps themselves where the TMA z-march serves them, the z faces by a
    copy).  One library call (``ps_diffusion3d_run_states``); ``graph=True`` replays its
    launches from the library's graph cache (keyed by the pointers: worth it when the same
    buffers come back, as in a loop of gradients).  ``temporal2=True`` (FP32): fused step
    pairs, bit for bit the same kept states (every = 1: pairs that write both states;
    every > 1: pairs that never step over a kept state)."""
    code = _code(T0)
    _same(T0, Ci)
    nx, ny, nz = _grid(T0)
    # the library takes the block as a base pointer and a stride in T0's elements
    if block.flat.dtype != T0.dtype or block.flat.device != T0.device or block.grids.shape != tuple(T0.shape):
        raise ValueError("the state block must hold grids of T0's shape, dtype and device")
    nslots = nt // every
    need = nslots + (2 if every > 1 and nt > 0 else 0)
    if len(block.grids) < need:
        raise ValueError(f"state block has {len(block.grids)} grids, needs {need}")
    slot = ctypes.c_int(0)
    check(_lib.load().ps_diffusion3d_run_states(
        _field(T0, "T0", code), block.ptr(), block.stride, int(every), _field(Ci, "Ci", code), lam,
        dt, *inv_spacing, nx, ny, nz, int(nt), code,
        (_lib.PS_RUN_CI_SCALED if ci_scaled else 0) | (_lib.PS_RUN_GRAPH if graph else 0)
        | (_lib.PS_RUN_TEMPORAL2 if temporal2 else 0), _stream(T0), ctypes.byref(slot)))
    s = slot.value
    if s == -3:
        return T0
    return block.grids[s] if s >= 0 else block.grids[nslots + (-1 - s)]


def run(T, T2, Ci, lam: float, dt: float, inv_spacing, nt: int, *, comp=None, graph=False,
        native_f64=False, ci_scaled=False, temporal2=False) -> torch.Tensor:
    """Fig. 1 time loop on the buffer pair (T, T2); returns the tensor holding T(nt).

    ``temporal2=True`` runs the steps in fused pairs (FP32, or FP64 with
    ``ci_scaled``); the result is bit for bit the same.  ``comp`` (FP32): the two
    correction fields of :func:`compensation_fields`; the steps are the compensated
    two-float steps and the result's correction ends in ``comp[nt % 2]``."""
    code = _code(T)
    _same(T, T2, Ci)
    nx, ny, nz = _grid(T)
    flags = 0
    if graph:
        flags |= _lib.PS_RUN_GRAPH
    if comp is not None:
        flags |= _lib.PS_RUN_COMPENSATED
        if tuple(comp.shape) != (2,) + tuple(T.shape) or comp.device != T.device:
            raise ValueError("comp must hold two correction fields: shape (2,) + T.shape "
                             "(see compensation_fields)")
    if native_f64:
        flags |= _lib.PS_RUN_NATIVE_F64
    if ci_scaled:
        flags |= _lib.PS_RUN_CI_SCALED
    if temporal2:
        flags |= _lib.PS_RUN_TEMPORAL2
    odd = ctypes.c_int(0)
    check(_lib.load().ps_diffusion3d_run_ex(
        _field(T, "T", code), _field(T2, "T2", code),
        _field(comp, "comp", PS_F32) if comp is not None else None, _field(Ci, "Ci", code), lam,
        dt, *inv_spacing, nx, ny, nz, int(nt), code, flags, _stream(T), ctypes.byref(odd)))
    return T2 if odd.value else T


def adjoint(Tbar, Cibar, ybar, T, Ci, lam: float, dt: float, inv_spacing, *,
            ci_scaled: bool = False) -> None:
    """Transposed step: Tbar := M^T ybar; Cibar += dt*lam*ybar*Lap(T) (interior).

    ``ci_scaled=True``: ``Ci`` is the pre-scaled field of :func:`scale_ci` and
    ``Cibar`` accumulates dL/dCs = ybar * L(T) (L = neighbour sum - 6 centre).
    """
    code = _code(T)
    _same(T, Tbar, Cibar, ybar, Ci)
    nx, ny, nz = _grid(T)
    check(_lib.load().ps_diffusion3d_adjoint_ex(
        _field(Tbar, "Tbar", code), _field(Cibar, "Cibar", code), _field(ybar, "ybar", code),
        _field(T, "T", code), _field(Ci, "Ci", code), lam, dt, *inv_spacing, nx, ny, nz, code,
        _lib.PS_RUN_CI_SCALED if ci_scaled else 0, _stream(T)))


def _grid2d(t: torch.Tensor):
    if t.dim() != 2:
        raise ValueError("2-D fields must have shape (ny, nx)")
    ny, nx = t.shape
    return nx, ny


def step2d(T2, T, Ci, lam: float, dt: float, inv_spacing: Sequence[float], *,
           ci_scaled: bool = False) -> None:
    """One step of the 2-D form of Fig. 1 (z term dropped) on (ny, nx) fields."""
    code = _code(T)
    _same(T, T2, Ci)
    nx, ny = _grid2d(T)
    check(_lib.load().ps_diffusion2d_step(_field(T2, "T2", code), _field(T, "T", code), _field(Ci, "Ci", code),
                                          lam, dt, inv_spacing[0], inv_spacing[1], nx, ny, code,
                                          _lib.PS_RUN_CI_SCALED if ci_scaled else 0, _stream(T)))


def run2d(T, T2, Ci, lam: float, dt: float, inv_spacing: Sequence[float], nt: int, *,
          graph: bool = False, ci_scaled: bool = False) -> torch.Tensor:
    """nt steps of the 2-D form (T2's edges set to T's first); returns the buffer
    holding T(nt)."""
    code = _code(T)
    _same(T, T2, Ci)
    nx, ny = _grid2d(T)
    odd = ctypes.c_int(0)
    flags = (_lib.PS_RUN_GRAPH if graph else 0) | (_lib.PS_RUN_CI_SCALED if ci_scaled else 0)
    check(_lib.load().ps_diffusion2d_run(_field(T, "T", code), _field(T2, "T2", code), _field(Ci, "Ci", code),
                                         lam, dt, inv_spacing[0], inv_spacing[1], nx, ny, int(nt), code, flags,
                                         _stream(T), ctypes.byref(odd)))
    return T2 if odd.value else T


def stable_dt2d(Ci, lam: float = 1.0, lengths=(1.0, 1.0)) -> float:
    """dt for the 2-D form: min(dx^2, dy^2)/lam/maximum(Ci)/4.1 (Fig. 1's rule with the
    2-D bound 4 in place of 6; ``ps_diffusion2d_stable_dt``, maximum(Ci) on the GPU)."""
    code = _code(Ci)
    nx, ny = _grid2d(Ci)
    v = ctypes.c_double(0.0)
    check(_lib.load().ps_diffusion2d_stable_dt(ctypes.byref(v), _field(Ci, "Ci", code), nx, ny, lam,
                                               lengths[0], lengths[1], code,
                                               workspace(Ci.device).data_ptr(), _stream(Ci)))
    return v.value


def adjoint2(Tbar, Cibar, ybar, T_first, T_second, Ci, lam: float, dt: float, inv_spacing) -> None:
    """Two transposed steps in one pass (FP32): with ybar = dL/dT_{t+2} and the
    states T_first = T_{t+1}, T_second = T_t, Tbar := dL/dT_t and Cibar accumulates
    both steps' terms, bit for bit two :func:`adjoint` calls."""
    code = _code(T_first)
    _same(T_first, T_second, Tbar, Cibar, ybar, Ci)
    nx, ny, nz = _grid(T_first)
    check(_lib.load().ps_diffusion3d_adjoint2_ex(
        _field(Tbar, "Tbar", code), _field(Cibar, "Cibar", code), _field(ybar, "ybar", code),
        _field(T_first, "T_first", code), _field(T_second, "T_second", code), _field(Ci, "Ci", code),
        lam, dt, *inv_spacing, nx, ny, nz, code, 0, _stream(T_first)))


def adjoint2_supported(T) -> bool:
    """Whether :func:`adjoint2` takes fields shaped and typed like ``T``."""
    return T.dtype == torch.float32 and T.shape[2] % 4 == 0


def maximum_async(A, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """max(A) into a 0-dim float64 device tensor (no synchronization)."""
    code = _code(A)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=A.device)
    check(_lib.load().ps_maximum_async(out.data_ptr(), _field(A, "A", code), A.numel(), code,
                                       workspace(A.device).data_ptr(), _stream(A)))
    return out


def maximum(A) -> float:
    """``maximum(A)`` returned to the host (synchronizes the stream)."""
    code = _code(A)
    v = ctypes.c_double(0.0)
    check(_lib.load().ps_maximum(ctypes.byref(v), _field(A, "A", code), A.numel(), code,
                                 workspace(A.device).data_ptr(), _stream(A)))
    return v.value


def stable_dt(Ci, lam: float = 1.0, lengths=(1.0, 1.0, 1.0)) -> float:
    """Fig. 1: ``dt = min(dx^2,dy^2,dz^2)/lam/maximum(Ci)/6.1`` (maximum on the GPU)."""
    code = _code(Ci)
    nx, ny, nz = _grid(Ci)
    v = ctypes.c_double(0.0)
    check(_lib.load().ps_diffusion3d_stable_dt(ctypes.byref(v), _field(Ci, "Ci", code), nx, ny, nz,
                                               lam, *lengths, code,
                                               workspace(Ci.device).data_ptr(), _stream(Ci)))
    return v.value


class SolvePipeline:
    """End-to-end solves of many problems of one shape, with the host copies hidden
    behind the computation.

    Each :meth:`submit` does what :func:`solve` does for one problem - copy T0 and
    Ci in from pinned host memory, dt from maximum(Ci) on the GPU, the pre-scaled
    coefficient (FP64, equal spacings), the nt steps (cached CUDA graph), copy
    T(nt) out to ``out_host`` - but the copies in run on their own stream into one
    of two device buffer sets and the copy out on a third stream, so that the
    inputs of problem i+1 arrive and the result of problem i-1 leaves while problem
    i computes.  Stream order and events keep every buffer's uses in order: problem
    i+2 overwrites a buffer set only after problem i's result has been copied out.
    ``submit`` returns the event recorded after the copy out (``out_host`` is valid
    once it has completed); :meth:`finish` waits for every submitted problem.  The
    host blocks only inside ``submit``, on the maximum(Ci) of its own problem.
    Call :meth:`finish` before reading results in bulk or dropping the pipeline
    (the buffers are released safely either way, but host tensors passed to
    ``submit`` must stay alive until their copies have completed).
    ``graph=True`` replays the nt steps from the library's graph cache, whose key
    holds dt: worth it only for small grids whose problems share dt (each new dt
    captures a graph); by default the steps are launched from the library's loop,
    which keeps the GPU fed whenever a step takes longer than a launch.
    """

    def __init__(self, shape, dtype, lam: float, inv_spacing, nt: int, *, device="cuda",
                 graph: bool = False, lengths=(1.0, 1.0, 1.0)):
        self.lam, self.inv, self.nt, self.graph, self.lengths = lam, tuple(inv_spacing), int(nt), graph, lengths
        self.device = torch.device(device)
        self.sets = [tuple(torch.empty(shape, dtype=dtype, device=self.device) for _ in range(3))
                     for _ in range(2)]
        self.s_in = torch.cuda.Stream(self.device)
        self.s_run = torch.cuda.Stream(self.device)
        self.s_out = torch.cuda.Stream(self.device)
        # the buffers are allocated on the caller's stream but used on the three streams:
        # tell the caching allocator, so that a pipeline dropped with work still queued
        # does not hand its blocks to a new allocation before that work completes
        for bufs in self.sets:
            for t in bufs:
                for st in (self.s_in, self.s_run, self.s_out):
                    t.record_stream(st)
        self.freed = [None, None]  # per set: event after its last result was copied out
        self.count = 0
        self.scaled = dtype == torch.float64 and self.inv[0] == self.inv[1] == self.inv[2]

    @staticmethod
    def check_host(shape, dtype, **tensors) -> None:
        """Host tensors of a submit: CPU tensors of the pipeline's exact shape and dtype
        (a copy would otherwise broadcast or convert silently)."""
        for name, t in tensors.items():
            if t.device.type != "cpu":
                raise ValueError(f"{name} must be a host (CPU) tensor, pinned for overlap")
            if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
                raise ValueError(f"{name} has shape {tuple(t.shape)} and dtype {t.dtype}; "
                                 f"the pipeline takes {tuple(shape)} {dtype}")

    def submit(self, T0_host: torch.Tensor, Ci_host: torch.Tensor, out_host: torch.Tensor):
        self.check_host(self.sets[0][0].shape, self.sets[0][0].dtype, T0_host=T0_host, Ci_host=Ci_host,
                        out_host=out_host)
        k = self.count % 2
        T, T2, Ci = self.sets[k]
        with torch.cuda.stream(self.s_in):
            if self.freed[k] is not None:
                self.s_in.wait_event(self.freed[k])
            # Ci first: dt and the scaled coefficient are formed while T arrives
            Ci.copy_(Ci_host, non_blocking=True)
            ci_arrived = torch.cuda.Event()
            ci_arrived.record(self.s_in)
            T.copy_(T0_host, non_blocking=True)
            arrived = torch.cuda.Event()
            arrived.record(self.s_in)
        with torch.cuda.stream(self.s_run):
            self.s_run.wait_event(ci_arrived)
            dt = stable_dt(Ci, self.lam, self.lengths)  # waits for this stream only
            if self.scaled:
                scale_ci(Ci, self.lam, dt, self.inv, out=Ci)
            self.s_run.wait_event(arrived)
            res = run(T, T2, Ci, self.lam, dt, self.inv, self.nt, graph=self.graph, ci_scaled=self.scaled)
            done = torch.cuda.Event()
            done.record(self.s_run)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(done)
            out_host.copy_(res, non_blocking=True)
            out = torch.cuda.Event()
            out.record(self.s_out)
        self.freed[k] = out
        self.count += 1
        return out

    def finish(self) -> None:
        for s in (self.s_in, self.s_run, self.s_out):
            s.synchronize()


def dot(A, B, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """sum(A*B) accumulated in FP64, as a 0-dim device tensor."""
    code = _code(A)
    _same(A, B)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=A.device)
    check(_lib.load().ps_dot(out.data_ptr(), _field(A, "A", code), _field(B, "B", code), A.numel(),
                             code, workspace(A.device).data_ptr(), _stream(A)))
    return out


def half_sq_dist(A, B, residual: Optional[torch.Tensor] = None,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """L = 1/2 ||A - B||^2 in FP64 (0-dim device tensor); optionally residual := A - B."""
    code = _code(A)
    _same(A, B)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=A.device)
    rptr = None
    if residual is not None:
        _same(A, residual)
        rptr = _field(residual, "residual", code)
    check(_lib.load().ps_half_sq_dist(out.data_ptr(), rptr, _field(A, "A", code),
                                      _field(B, "B", code), A.numel(), code,
                                      workspace(A.device).data_ptr(), _stream(A)))
    return out


def to_deviation(T: torch.Tensor, t_ref: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP32 deviation field ``(float)(T - t_ref)`` of an FP64 field."""
    if out is None:
        out = torch.empty(T.shape, dtype=torch.float32, device=T.device)
    check(_lib.load().ps_to_deviation(_field(out, "D", PS_F32), _field(T, "T", PS_F64), t_ref,
                                      T.numel(), _stream(T)))
    return out


def from_deviation(D: torch.Tensor, t_ref: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP64 field ``(double)D + t_ref`` from an FP32 deviation field."""
    if out is None:
        out = torch.empty(D.shape, dtype=torch.float64, device=D.device)
    check(_lib.load().ps_from_deviation(_field(out, "T", PS_F64), _field(D, "D", PS_F32), t_ref,
                                        D.numel(), _stream(D)))
    return out


def to_deviation_pair(T: torch.Tensor, t_ref: float):
    """Two-float deviation (D, E) of an FP64 field: D = (float)(T - t_ref), E the FP32
    rounding of what D misses (``ps_to_deviation_pair``)."""
    D = torch.empty(T.shape, dtype=torch.float32, device=T.device)
    E = torch.empty_like(D)
    check(_lib.load().ps_to_deviation_pair(_field(D, "D", PS_F32), _field(E, "E", PS_F32),
                                           _field(T, "T", PS_F64), t_ref, T.numel(), _stream(T)))
    return D, E


def from_deviation_pair(D: torch.Tensor, E: torch.Tensor, t_ref: float) -> torch.Tensor:
    """FP64 field ``(D + E) + t_ref`` of a two-float state."""
    _same(D, E)
    out = torch.empty(D.shape, dtype=torch.float64, device=D.device)
    check(_lib.load().ps_from_deviation_pair(_field(out, "T", PS_F64), _field(D, "D", PS_F32),
                                             _field(E, "E", PS_F32), t_ref, D.numel(), _stream(D)))
    return out


def to_f32(A: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FP32 copy of an FP64 coefficient field (one rounding per element)."""
    return to_deviation(A, 0.0, out)


def _pitch(t: torch.Tensor, name: str) -> int:
    """Row pitch (elements) of a field: contiguous, or a view whose rows are
    `pitch` elements apart and whose planes are pitch*ny apart (see
    :func:`pitched_empty`)."""
    if t.dim() != 3:
        raise ValueError("fields must have shape (nz, ny, nx)")
    nz, ny, nx = t.shape
    if t.is_contiguous():
        return nx
    sz, sy, sx = t.stride()
    if sx != 1 or sy < nx or sz != sy * ny:
        raise ValueError(f"{name} must be contiguous or padded along x only (rows {sy} apart, planes rows*ny)")
    return sy


def pitched_empty(shape, dtype=torch.float64, device="cuda") -> torch.Tensor:
    """Uninitialised (nz, ny, nx) field whose rows start on 16-byte boundaries:
    a view of an (nz, ny, pitch) block, pitch = nx rounded up to 16 bytes.  Its
    rows can be staged by TMA whatever nx is (the batched z-march needs this)."""
    nz, ny, nx = shape
    per = 16 // torch.empty((), dtype=dtype).element_size()
    pitch = -(-nx // per) * per
    return torch.empty((nz, ny, pitch), dtype=dtype, device=device)[:, :, :nx]


def pitched_copy(t: torch.Tensor) -> torch.Tensor:
    """A copy of field ``t`` in the layout of :func:`pitched_empty`."""
    out = pitched_empty(tuple(t.shape), t.dtype, t.device)
    out.copy_(t)
    return out


class Batch:
    """Many independent problems stepped together, one launch per step.

    ``problems`` is a list of dicts with keys ``T, T2, Ci`` (CUDA tensors of
    one dtype, any cubic or non-cubic shape; contiguous, or padded along x as
    :func:`pitched_empty` makes them, the three with one pitch), ``lam``,
    ``dt`` and ``inv_spacing``, and optionally ``tile`` = (tile_x, tile_y,
    tile_z) for that problem's work items (see ``tuner.tuned_batch``).  T2's
    boundary must equal T's (e.g. ``T2 = T.clone()``).

    ``kernel``: "auto" (the TMA z-march when every problem can take it, else
    the column march), "zmarch" or "column".  ``ci_scaled``: FP64 problems
    whose ``Ci`` holds the pre-scaled ``dt*lam*_dx^2*Ci`` of :func:`scale_ci`
    (equal spacings; z-march).  ``temporal2``: :meth:`run` steps in fused pairs
    (temporal blocking of depth 2; z-march, FP32 or FP64 with ``ci_scaled``).
    ``prescale`` (default on): FP64 problems given with Ci as it is are stepped on
    the pre-scaled coefficient when every problem can take it (the z-march, equal
    spacings, dt*lam*_dx^2 > 0): the batch keeps its own copy Cs = dt*lam*_dx^2*Ci
    per problem, made at construction (``ps_diffusion3d_scale_ci``; a later change
    of Ci needs a new Batch), and each step costs one FP64 multiply-add per node,
    the arithmetic of :func:`solve` - a problem then equals its single run on that
    Cs bit for bit.  ``prescale=False`` keeps the kernel on Ci as given (two FP64
    products per node).  The chosen kernel is ``self.kernel``; ``self.prescaled``
    tells whether the batch steps on its own Cs.
    """

    KERNELS = {"auto": 0, "column": _lib.PS_BATCH_COLUMN, "zmarch": _lib.PS_BATCH_ZMARCH}

    @staticmethod
    def _prescalable(problems, kernel: str) -> bool:
        """FP64 problems that can all take the pre-scaled z-march."""
        if kernel == "column":
            return False
        for p in problems:
            T, inv = p["T"], p["inv_spacing"]
            if T.dtype != torch.float64 or not (inv[0] == inv[1] == inv[2]):
                return False
            if (_pitch(T, "T") * 8) % 16 != 0 or not (p["dt"] * p["lam"] * inv[0] * inv[0] > 0.0):
                return False
        return True

    @staticmethod
    def _scaled_copy(p) -> torch.Tensor:
        """Cs = dt*lam*_dx^2*Ci in a field of Ci's layout (the pitched block scaled whole)."""
        Ci = p["Ci"]
        nz, ny, nx = Ci.shape
        pitch = _pitch(Ci, "Ci")
        Cs = torch.empty((nz, ny, pitch), dtype=Ci.dtype, device=Ci.device)
        block = Ci.as_strided((nz, ny, pitch), (ny * pitch, pitch, 1)) if pitch != nx else Ci
        scale_ci(block, p["lam"], p["dt"], p["inv_spacing"], out=Cs)
        return Cs[:, :, :nx] if pitch != nx else Cs

    def __init__(self, problems, tile=(0, 0, 0), kernel: str = "auto", ci_scaled: bool = False,
                 temporal2: bool = False, prescale: bool = True):
        if not problems:
            raise ValueError("empty batch")
        if kernel not in self.KERNELS:
            raise ValueError(f"kernel must be one of {sorted(self.KERNELS)}")
        lib = _lib.load()
        self.code = _code(problems[0]["T"])
        self.device = problems[0]["T"].device
        self.prescaled = bool(prescale and not ci_scaled and self._prescalable(problems, kernel))
        if self.prescaled:
            problems = [dict(p, Ci=self._scaled_copy(p)) for p in problems]
            ci_scaled = True
        self.problems = problems
        arr = (_lib.PsProblem * len(problems))()
        for q, p in enumerate(problems):
            _same(p["T"], p["T2"], p["Ci"])
            nx, ny, nz = _grid(p["T"])
            pitches = {_pitch(p[k], k) for k in ("T", "T2", "Ci")}
            if len(pitches) != 1:
                raise ValueError(f"problem {q}: T, T2 and Ci must share one row pitch")
            for k in ("T", "T2", "Ci"):
                if not p[k].is_cuda or _code(p[k]) != self.code or p[k].device != self.device:
                    raise TypeError(f"problem {q}: {k} must be a CUDA tensor of the batch's dtype "
                                    "on the batch's device")
            tx, ty, tz = p.get("tile", (0, 0, 0))
            arr[q] = _lib.PsProblem(p["T"].data_ptr(), p["T2"].data_ptr(), p["Ci"].data_ptr(),
                                    p["lam"], p["dt"], *p["inv_spacing"], nx, ny, nz, tx, ty, tz,
                                    pitches.pop())
        flags = (self.KERNELS[kernel] | (_lib.PS_BATCH_CI_SCALED if ci_scaled else 0) |
                 (_lib.PS_BATCH_TEMPORAL2 if temporal2 else 0))
        self.temporal2 = temporal2
        nbytes = lib.ps_batch_table_bytes_ex(arr, len(problems), self.code, *tile, flags)
        # 64-byte aligned host buffer (the z-march table embeds tensor maps)
        raw = (ctypes.c_char * (nbytes + 64))()
        off = (-ctypes.addressof(raw)) % 64
        host = (ctypes.c_char * max(nbytes, 1)).from_buffer(raw, off)
        nitems = ctypes.c_int64(0)
        check(lib.ps_batch_table_fill_ex(host, nbytes, arr, len(problems), self.code, *tile, flags,
                                         ctypes.byref(nitems)))
        self._host_raw = raw  # keeps `host` alive: the step and run calls read its header
        self.host = host
        self.nitems = nitems.value
        self.tile = tile
        self.kernel = "zmarch" if lib.ps_batch_table_kernel(host) == 1 else "column"
        cpu = torch.frombuffer(bytearray(host.raw), dtype=torch.uint8)
        self.table = cpu.to(self.device)
        torch.cuda.current_stream(self.device).synchronize()

    def step(self, parity: int) -> None:
        check(_lib.load().ps_diffusion3d_batch_step_ex(self.table.data_ptr(), self.host, int(parity),
                                                       torch.cuda.current_stream(self.device).cuda_stream))

    def step2(self, parity: int) -> None:
        """Two steps in one launch (a batch built with ``temporal2``)."""
        check(_lib.load().ps_diffusion3d_batch_step2_ex(self.table.data_ptr(), self.host, int(parity),
                                                        torch.cuda.current_stream(self.device).cuda_stream))

    def run(self, nt: int, graph: bool = True) -> None:
        """nt steps (fused pairs when built with ``temporal2``); problem p's state
        ends in T2 when nt is odd, in T when even."""
        flags = (_lib.PS_RUN_GRAPH if graph else 0) | (_lib.PS_RUN_TEMPORAL2 if self.temporal2 else 0)
        check(_lib.load().ps_diffusion3d_batch_run_ex(self.table.data_ptr(), self.host, int(nt), flags,
                                                      torch.cuda.current_stream(self.device).cuda_stream))

    def result(self, q: int, nt: int) -> torch.Tensor:
        p = self.problems[q]
        return p["T2"] if nt & 1 else p["T"]


def clear_graph_cache() -> None:
    check(_lib.load().ps_clear_graph_cache())


def graph_cache_size() -> int:
    """Graphs held by the library's cache (at most 256, least recently used evicted)."""
    return int(_lib.load().ps_graph_cache_size())


def set_launch_override(name: str, value: int) -> int:
    """Set a launch-shape override (``ps_set_launch_override``): ``name`` is one of
    ``kchunk, kchunk2, adj_kchunk, chunk2d`` (planes or rows per CTA, 0 = the library's
    rule) or ``adj_plain, f64_px2, step_plain`` (0/1).  Returns the previous value.  The forward
    steps' shapes give bit for bit the same fields; the FP64 transposed step's z-chunk sets
    its fixed-point scale and so can change low-order bits within tolerance.  A change
    empties the graph cache."""
    lib = _lib.load()
    which = _lib.PS_OVERRIDE[name]
    old = ctypes.c_int(0)
    check(lib.ps_get_launch_override(which, ctypes.byref(old)))
    check(lib.ps_set_launch_override(which, int(value)))
    return old.value


class launch_override:
    """Context manager: ``with launch_override(kchunk=7): ...`` sets overrides for the
    block and restores the previous values after it."""

    def __init__(self, **values):
        self.values = values
        self.saved = {}

    def __enter__(self):
        for name, v in self.values.items():
            self.saved[name] = set_launch_override(name, v)
        return self

    def __exit__(self, *exc):
        for name, v in self.saved.items():
            set_launch_override(name, v)
        return False


def step_kernel_name(T2, T, Ci, lam, dt, inv_spacing, ci_scaled=False, temporal2=False) -> str:
    """Name of the kernel that :func:`step` (or, with ``temporal2``, a fused pair
    of :func:`run`) launches for these arguments."""
    code = _code(T)
    nx, ny, nz = _grid(T)
    flags = (_lib.PS_RUN_CI_SCALED if ci_scaled else 0) | (_lib.PS_RUN_TEMPORAL2 if temporal2 else 0)
    name = _lib.load().ps_diffusion3d_step_kernel(T2.data_ptr(), T.data_ptr(), Ci.data_ptr(), lam,
                                                  dt, *inv_spacing, nx, ny, nz, code, flags)
    return name.decode()


KERNEL_SOURCES = {
    "k_zmarch": ["paper_2211_15634_gb300/csrc/zmarch.cu", "paper_2211_15634_gb300/csrc/zmarch_tile.cuh",
                 "paper_2211_15634_gb300/csrc/zmarch.h", "paper_2211_15634_gb300/csrc/emu64.cuh",
                 "paper_2211_15634_gb300/csrc/node.cuh", "paper_2211_15634_gb300/csrc/tma.cuh",
                 "paper_2211_15634_gb300/csrc/pdl.cuh"],
    "k_zmarch2": ["paper_2211_15634_gb300/csrc/zmarch2.cu", "paper_2211_15634_gb300/csrc/zmarch2_tile.cuh",
                  "paper_2211_15634_gb300/csrc/emu64.cuh",
                  "paper_2211_15634_gb300/csrc/node.cuh", "paper_2211_15634_gb300/csrc/tma.cuh",
                  "paper_2211_15634_gb300/csrc/pdl.cuh"],
    "k_step_basic_emu": ["paper_2211_15634_gb300/csrc/stencil_basic.cuh",
                         "paper_2211_15634_gb300/csrc/emu64.cuh"],
    "k_step_basic": ["paper_2211_15634_gb300/csrc/stencil_basic.cuh"],
}


def step_kernel_sources(name: str):
    """Source files of a step kernel, relative to the repository root."""
    return KERNEL_SOURCES[name.split("<")[0]]


def device_error(clear: bool = False) -> int:
    """Device-side error flags (bit 0: a bounded pipeline wait timed out)."""
    v = ctypes.c_uint(0)
    check(_lib.load().ps_device_error(ctypes.byref(v), int(clear)))
    return v.value


def solve(T0_host: torch.Tensor, Ci_host: torch.Tensor, lam: float, dt: Optional[float],
          inv_spacing, nt: int, *, device="cuda", graph: bool = True,
          out_host: Optional[torch.Tensor] = None, buffers=None,
          lengths=(1.0, 1.0, 1.0)) -> torch.Tensor:
    """End to end: host fields in (pinned CPU tensors), T(nt) back on the host.

    ``dt=None`` takes Fig. 1's stable step from maximum(Ci) (reduced on the
    GPU).  ``buffers`` may hold preallocated device tensors ``(T, T2, Ci)``.
    On FP64 grids with equal spacings the device ``Ci`` ends up holding the
    pre-scaled coefficient of :func:`scale_ci`.
    """
    if buffers is None:
        T = torch.empty(T0_host.shape, dtype=T0_host.dtype, device=device)
        T2 = torch.empty_like(T)
        Ci = torch.empty(Ci_host.shape, dtype=Ci_host.dtype, device=device)
    else:
        T, T2, Ci = buffers
    T.copy_(T0_host, non_blocking=True)
    Ci.copy_(Ci_host, non_blocking=True)
    if dt is None:
        dt = stable_dt(Ci, lam, lengths)
    scaled = (T.dtype == torch.float64 and inv_spacing[0] == inv_spacing[1] == inv_spacing[2])
    if scaled:  # fold dt*lam*_dx^2 into the coefficient field once per solve
        scale_ci(Ci, lam, dt, inv_spacing, out=Ci)
    res = run(T, T2, Ci, lam, dt, inv_spacing, nt, graph=graph, ci_scaled=scaled)
    if out_host is None:
        out_host = torch.empty(T0_host.shape, dtype=T0_host.dtype, pin_memory=True)
    out_host.copy_(res, non_blocking=True)
    torch.cuda.current_stream(T.device).synchronize()
    return out_host
