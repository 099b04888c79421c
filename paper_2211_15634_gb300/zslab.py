"""One problem split into z-slabs over several ranks, with a one-plane halo exchange
per step and the boundary planes stepped first so that the exchange hides behind
the interior (the decomposition of the paper's multi-GPU runs: ImplicitGlobalGrid
with communication hidden behind computation, Sect. Approach and Results).

Rank r of R owns a contiguous range [z0, z1) of the global interior planes 1..nz-2
(ranges as even as possible, or given).  Its local fields hold nz_loc = z1 - z0 + 2
planes: local plane 0 is global plane z0 - 1 and local plane nz_loc - 1 is global
plane z1 - the neighbours' last / first owned planes (halos) or the global z
boundary.  A local step with the library's kernel writes exactly the owned planes
(the local z faces are the kernel's fixed boundary), so after every step each rank
sends its first owned plane down and its last one up and receives the halos of the
new state; the global x/y boundaries are local boundaries too.  Each node is stepped
by the same kernel arithmetic as in a single-grid run, so the decomposed run gives
the single-grid result bit for bit.

Exchange transports (``HaloExchange``): ``"device"`` sends the planes' device memory
through ``torch.distributed`` point-to-point calls (NCCL: copies into the receiving
GPU's own memory); ``"host"`` stages them through pinned host memory (any backend,
e.g. gloo), and the interior step still runs on the GPU meanwhile.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import torch

from . import api


def split_planes(nz: int, world: int, sizes: Optional[Sequence[int]] = None) -> List[tuple]:
    """Owned global plane ranges [z0, z1) of the interior planes 1..nz-2 for each
    rank: ``sizes`` (each >= 1, summing to nz - 2) or as even as possible."""
    inner = nz - 2
    if world < 1 or inner < world:
        raise ValueError(f"cannot split {inner} interior planes over {world} ranks")
    if sizes is None:
        q, r = divmod(inner, world)
        sizes = [q + (1 if i < r else 0) for i in range(world)]
    sizes = [int(s) for s in sizes]
    if len(sizes) != world or any(s < 1 for s in sizes) or sum(sizes) != inner:
        raise ValueError(f"sizes {sizes} must be {world} values >= 1 summing to {inner}")
    out, z = [], 1
    for s in sizes:
        out.append((z, z + s))
        z += s
    return out


class ZSlab:
    """The slab of one rank: global size (nz, ny, nx), owned planes [z0, z1)."""

    def __init__(self, shape, rank: int, world: int, sizes=None):
        self.nz, self.ny, self.nx = (int(v) for v in shape)
        self.rank, self.world = int(rank), int(world)
        self.ranges = split_planes(self.nz, self.world, sizes)
        self.z0, self.z1 = self.ranges[self.rank]
        self.nz_loc = self.z1 - self.z0 + 2

    @property
    def local_shape(self):
        return (self.nz_loc, self.ny, self.nx)

    @property
    def down(self) -> Optional[int]:
        """Rank holding the planes below (None at the global z = 0 boundary)."""
        return self.rank - 1 if self.rank > 0 else None

    @property
    def up(self) -> Optional[int]:
        return self.rank + 1 if self.rank < self.world - 1 else None

    def local_view(self, A_global: torch.Tensor) -> torch.Tensor:
        """This rank's planes z0-1 .. z1 of a global field (a view)."""
        return A_global[self.z0 - 1:self.z1 + 1]

    def owned(self, A_local: torch.Tensor) -> torch.Tensor:
        """The owned planes of a local field (a view)."""
        return A_local[1:self.nz_loc - 1]


class HaloExchange:
    """Plane exchange between neighbouring slabs after a step: the first owned plane
    of A goes down (it is the lower neighbour's top halo), the last one up; the halos
    of A are received.  ``transport``: "device" or "host" (see the module doc)."""

    def __init__(self, slab: ZSlab, like: torch.Tensor, transport: str = "device", group=None):
        import torch.distributed as dist
        self.dist = dist
        self.slab, self.group, self.transport = slab, group, transport
        if transport not in ("device", "host"):
            raise ValueError("transport must be 'device' or 'host'")
        plane = (slab.ny, slab.nx)
        if transport == "host":
            pin = like.is_cuda
            mk = lambda: torch.empty(plane, dtype=like.dtype, pin_memory=pin)  # noqa: E731
            self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()

    def _peer(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def start(self, A: torch.Tensor):
        """Post the exchange for field A (after its owned boundary planes are final on
        the current stream); returns a handle for :meth:`finish`."""
        s, d = self.slab, self.dist
        lo, hi = 1, s.nz_loc - 2  # first / last owned local planes
        ops = []
        if self.transport == "device":
            if s.down is not None:
                ops.append(d.P2POp(d.isend, A[lo], self._peer(s.down), self.group))
                ops.append(d.P2POp(d.irecv, A[0], self._peer(s.down), self.group))
            if s.up is not None:
                ops.append(d.P2POp(d.isend, A[hi], self._peer(s.up), self.group))
                ops.append(d.P2POp(d.irecv, A[s.nz_loc - 1], self._peer(s.up), self.group))
            works = d.batch_isend_irecv(ops) if ops else []
            return ("device", works, A)
        # host staging: the boundary planes come down once they are final
        if s.down is not None:
            self.send_lo.copy_(A[lo], non_blocking=True)
        if s.up is not None:
            self.send_hi.copy_(A[hi], non_blocking=True)
        ev = None
        if A.is_cuda:
            ev = torch.cuda.Event()
            ev.record()
        return ("host", ev, A)

    def finish(self, handle) -> None:
        """Complete the exchange: afterwards A's halo planes hold the neighbours'
        owned planes (in stream order on the current stream for "device")."""
        kind, h, A = handle
        s, d = self.slab, self.dist
        if kind == "device":
            for w in h:
                w.wait()
            return
        if h is not None:
            h.synchronize()  # the staged planes are on the host
        ops = []
        if s.down is not None:
            ops.append(d.P2POp(d.isend, self.send_lo, self._peer(s.down), self.group))
            ops.append(d.P2POp(d.irecv, self.recv_lo, self._peer(s.down), self.group))
        if s.up is not None:
            ops.append(d.P2POp(d.isend, self.send_hi, self._peer(s.up), self.group))
            ops.append(d.P2POp(d.irecv, self.recv_hi, self._peer(s.up), self.group))
        for w in (d.batch_isend_irecv(ops) if ops else []):
            w.wait()
        if s.down is not None:
            A[0].copy_(self.recv_lo, non_blocking=True)
        if s.up is not None:
            A[s.nz_loc - 1].copy_(self.recv_hi, non_blocking=True)


def default_step(T2, T, Ci, lam, dt, inv, ci_scaled=False):
    """One library step (the CUDA kernels) on a (sub-)volume."""
    api.step(T2, T, Ci, lam, dt, inv, ci_scaled=ci_scaled)


def run_slab(slab: ZSlab, exchange: Optional[HaloExchange], T: torch.Tensor, T2: torch.Tensor,
             Ci: torch.Tensor, lam: float, dt: float, inv, nt: int, *, ci_scaled: bool = False,
             overlap: bool = True, step: Callable = default_step) -> torch.Tensor:
    """nt steps of the decomposed problem on this rank's local fields (T, T2, Ci of
    ``slab.local_shape``; T's halos hold the neighbours' planes of the initial state,
    its local z faces the global boundary where there is no neighbour).  T2's
    boundary is set from T first (Fig. 1's ``T2 = copy(T)``).  ``overlap``: step the
    two owned boundary planes first, exchange them while the interior planes are
    stepped (needs two owned planes or more and plane offsets that keep 16-byte
    alignment; else the whole slab is stepped, then exchanged).  Returns the local field holding T(nt).
    ``step`` is the per-volume step (the library's kernel)."""
    n = slab.nz_loc
    api.copy_boundary(T2, T) if T.is_cuda else T2.copy_(T)
    plane_bytes = slab.ny * slab.nx * T.element_size()
    can_overlap = overlap and n >= 4 and plane_bytes % 16 == 0
    src, dst = T, T2
    for _ in range(nt):
        if can_overlap:
            # owned boundary planes first: local planes 1 and n-2 (3-plane views)
            step(dst[0:3], src[0:3], Ci[0:3], lam, dt, inv, ci_scaled=ci_scaled)
            step(dst[n - 3:n], src[n - 3:n], Ci[n - 3:n], lam, dt, inv, ci_scaled=ci_scaled)
            h = exchange.start(dst) if exchange is not None else None
            # interior planes 2 .. n-3 (a view of planes 1 .. n-2) while the halos travel
            if n >= 5:
                step(dst[1:n - 1], src[1:n - 1], Ci[1:n - 1], lam, dt, inv, ci_scaled=ci_scaled)
            if h is not None:
                exchange.finish(h)
        else:
            step(dst, src, Ci, lam, dt, inv, ci_scaled=ci_scaled)
            if exchange is not None:
                exchange.finish(exchange.start(dst))
        src, dst = dst, src
    return src
