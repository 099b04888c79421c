"""The failure path of the pipelined kernels without a GPU fault: a bounded wait on an
mbarrier that nothing arrives on gives up, reports through ps_device_error, and the
context stays usable."""
import time

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host
from paper_2211_15634_gb300 import _lib, api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    lib = _lib.load()
    api.device_error(clear=True)
    t0 = time.perf_counter()
    _lib.check(lib.ps_selftest_bounded_wait(4096, 1000, torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert api.device_error(clear=True) & 1
    assert elapsed < 5.0  # 4096 polls of at most 1 us each, plus the launch
    assert api.device_error() == 0
    # the next work runs normally
    T0, Ci, lam, dt, inv = problem(36, 20, 14)
    T = to_dev(T0)
    got = to_host(api.run(T, torch.empty_like(T), to_dev(Ci), lam, dt, inv, 5))
    assert rel_linf(got, oracle.run(T0, Ci, lam, dt, *inv, 5)) <= 1e-12
    assert api.device_error() == 0
