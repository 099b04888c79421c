"""maximum(A) returned to the host (Fig. 1's maximum(Ci), the input of dt): the
finishing kernel stores the value into a pinned, mapped host slot from a pool, so the
read-back waits for no copy engine.  The maximum is exact, so every result must equal
torch's maximum bit for bit: repeated calls, calls from several threads on their own
streams at once (each call holds its own slot), and a call made while a 1 GiB copy
to the host is in flight on another stream, which must return before that copy has
finished."""
import threading

import pytest
import torch

from paper_2211_15634_gb300 import api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_repeated_calls_are_exact(dtype):
    g = torch.Generator(device="cuda").manual_seed(5)
    for n in (1, 7, 1000, 1 << 20):
        A = torch.randn(n, device="cuda", dtype=dtype, generator=g)
        for _ in range(3):
            assert api.maximum(A) == float(A.max())


def test_concurrent_threads_each_on_their_own_stream():
    dev = torch.device("cuda", torch.cuda.current_device())
    fields = [torch.rand(3 << 18, device=dev, dtype=torch.float64) * (t + 1) for t in range(4)]
    expect = [float(A.max()) for A in fields]
    got = [[] for _ in fields]
    errors = []

    def worker(t):
        try:
            torch.cuda.set_device(dev)
            with torch.cuda.stream(torch.cuda.Stream(dev)):
                for _ in range(40):
                    got[t].append(api.maximum(fields[t]))
        except Exception as e:  # reported on the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(len(fields))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    assert not errors
    for t in range(len(fields)):
        assert got[t] == [expect[t]] * 40


def test_does_not_wait_for_a_copy_in_flight_on_another_stream():
    big = torch.ones(1 << 27, device="cuda", dtype=torch.float64)  # 1 GiB
    host = torch.empty(big.shape, dtype=big.dtype, pin_memory=True)
    A = torch.rand(1 << 16, device="cuda", dtype=torch.float64)
    expect = float(A.max())
    s_copy, s_red = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s_copy):
        host.copy_(big, non_blocking=True)
        done = torch.cuda.Event()
        done.record(s_copy)
    with torch.cuda.stream(s_red):
        v = api.maximum(A)
    in_flight = not done.query()
    done.synchronize()
    assert v == expect
    assert in_flight, "maximum() returned only after the 1 GiB copy on another stream had finished"
    assert float(host[-1]) == 1.0
