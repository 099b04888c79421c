"""The benchmark's multi-rank logic on CPU: two gloo ranks with different local
times agree on the slowest time, and the whole-job rate counts both replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank])
        rate = bench.whole_job_rate(1000.0, slowest, world)
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world, port = 2, _free_port()
    times = [0.5, 2.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [2.0, 2.0]
    assert all(abs(r[2] - 1000.0) < 1e-9 for r in res)  # 2 ranks x 1000 units / 2 s


def test_single_process_is_local():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0


@pytest.mark.parametrize("world", [2])
def test_reference_arm_only_rank0_prints(world, capsys, monkeypatch):
    """Under torchrun the reference arm runs on rank 0 only; other ranks exit 0."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", str(world))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
