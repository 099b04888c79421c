"""Z-slab decomposition of one problem with the library's step kernel: two ranks
(processes) share cuda:0 and exchange their halo planes through pinned host memory
with gloo after every step (the boundary planes are stepped first and the interior
steps while the planes travel).  No kernel waits on another rank: the ranks meet
only on the host.  The gathered field must equal the single-grid run bit for bit
and the FP64 oracle within 1e-12."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def fields(shape):
    from paper_2211_15634_gb300 import inputs
    nz, ny, nx = shape
    T0 = 1.7 + inputs.random_field(shape, 41, 0.0, 1.0)
    Ci = inputs.ci_random(nx, ny, nz)
    d = 1.0 / (max(shape) - 1)
    dt = d * d / Ci.max() / 6.1
    return T0, Ci, dt, (1.0 / d,) * 3


def _rank(rank, world, port, shape, sizes, nt, scaled, overlap, out):
    import torch.distributed as dist

    from paper_2211_15634_gb300 import api, zslab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        T0, Ci, dt, inv = fields(shape)
        slab = zslab.ZSlab(shape, rank, world, sizes)
        T = torch.from_numpy(np.ascontiguousarray(T0[slab.z0 - 1:slab.z1 + 1])).cuda()
        C = torch.from_numpy(np.ascontiguousarray(Ci[slab.z0 - 1:slab.z1 + 1])).cuda()
        if scaled:
            C = api.scale_ci(C, 1.0, dt, inv)
        T2 = torch.empty_like(T)
        ex = zslab.HaloExchange(slab, T, transport="host")
        res = zslab.run_slab(slab, ex, T, T2, C, 1.0, dt, inv, nt, ci_scaled=scaled, overlap=overlap)
        owned = slab.owned(res).cpu().numpy()
        assert api.device_error() == 0
        parts = [None] * world
        dist.all_gather_object(parts, (slab.z0, owned))
        if rank == 0:
            full = T0.copy()
            for z0, a in parts:
                full[z0:z0 + a.shape[0]] = a
            out.put(full)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,sizes,nt,scaled,overlap", [
    ((37, 29, 64), [14, 21], 9, True, True),
    ((37, 29, 64), None, 6, False, True),
    ((20, 16, 66), [2, 16], 5, True, False),
])
def test_two_slabs_equal_the_single_grid_run(shape, sizes, nt, scaled, overlap):
    import oracle
    from paper_2211_15634_gb300 import api
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shape, sizes, nt, scaled, overlap, q))
             for r in range(world)]
    for p in procs:
        p.start()
    full = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    T0, Ci, dt, inv = fields(shape)
    T = torch.from_numpy(T0).cuda()
    C = torch.from_numpy(Ci).cuda()
    if scaled:
        C = api.scale_ci(C, 1.0, dt, inv)
    single = api.run(T, torch.empty_like(T), C, 1.0, dt, inv, nt, ci_scaled=scaled).cpu().numpy()
    assert np.array_equal(full, single)
    ref = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
    assert np.max(np.abs(full - ref)) <= 1e-12 * np.max(np.abs(ref))
