"""Z-slab decomposition of one problem (zslab.py) on CPU with gloo ranks: the plane
partition, the halo exchange after every step (both transports) and the
boundary-first order of the steps.  Each rank steps its slab with the FP64 oracle's
step on CPU tensors (the library's kernel needs a GPU; the GPU form of this test is
test_gpu_zslab.py), so the decomposed run must equal the oracle's whole-grid run
bit for bit: every node sees the same seven values and the same arithmetic."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2211_15634_gb300 import zslab


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_planes_even_uneven_and_invalid():
    assert zslab.split_planes(12, 3) == [(1, 5), (5, 8), (8, 11)]
    assert zslab.split_planes(9, 2, sizes=[2, 5]) == [(1, 3), (3, 8)]
    assert zslab.split_planes(3, 1) == [(1, 2)]
    for args in ((4, 3), (9, 2, [3, 3]), (9, 2, [0, 7])):
        with pytest.raises(ValueError):
            zslab.split_planes(*args)
    s = zslab.ZSlab((9, 4, 6), 1, 2, sizes=[2, 5])
    assert (s.z0, s.z1, s.nz_loc, s.down, s.up) == (3, 8, 7, 0, None)
    assert s.local_shape == (7, 4, 6)


def _oracle_step(T2, T, Ci, lam, dt, inv, ci_scaled=False):
    import oracle
    oracle.step(T2.numpy(), T.numpy(), Ci.numpy(), lam, dt, *inv)


def _rank(rank, world, port, shape, sizes, nt, transport, overlap, out):
    import torch.distributed as dist

    import oracle
    from paper_2211_15634_gb300 import inputs
    oracle.build()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nz, ny, nx = shape
        T0 = torch.from_numpy(1.7 + inputs.random_field(shape, 31, 0.0, 1.0))
        Ci = torch.from_numpy(inputs.ci_random(nx, ny, nz))
        dx, dy, dz = inputs.spacing(nx, ny, nz)
        dt = min(dx * dx, dy * dy, dz * dz) / float(Ci.max()) / 6.1
        inv = inputs.inverse_spacing(nx, ny, nz)
        slab = zslab.ZSlab(shape, rank, world, sizes)
        T = slab.local_view(T0).clone()
        C = slab.local_view(Ci).clone()
        T2 = torch.empty_like(T)
        ex = zslab.HaloExchange(slab, T, transport=transport)
        res = zslab.run_slab(slab, ex, T, T2, C, 1.0, dt, inv, nt, overlap=overlap, step=_oracle_step)
        owned = slab.owned(res).contiguous()
        parts = [None] * world
        dist.all_gather_object(parts, (slab.z0, owned.numpy()))
        if rank == 0:
            full = T0.numpy().copy()
            for z0, a in parts:
                full[z0:z0 + a.shape[0]] = a
            ref = oracle.run(T0.numpy(), Ci.numpy(), 1.0, dt, *inv, nt)
            out.put(bool(np.array_equal(full, ref)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,sizes,nt,transport,overlap", [
    (2, (17, 9, 12), None, 5, "device", True),
    (2, (17, 9, 12), [3, 12], 4, "host", True),
    (2, (17, 9, 12), [11, 4], 3, "device", False),
    (3, (14, 7, 8), [1, 6, 5], 6, "host", True),
    (3, (14, 7, 8), None, 7, "device", True),
])
def test_decomposed_run_equals_whole_grid(world, shape, sizes, nt, transport, overlap):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, sizes, nt, transport, overlap, q))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert q.get(timeout=10) is True
