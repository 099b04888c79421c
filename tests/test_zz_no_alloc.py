"""ps_dot_static, the dot product that allocates nothing, against ps_dot.

Some callers cannot allocate device memory (a plugin inside a host program
that owns every device allocation, or a loop that must not allocate while it
runs).  ps_dot_static keeps its partial sums in an array inside the library
image instead of a caller workspace.  These tests call it through the C ABI
and compare it with ps_dot, the workspace-based entry point, within the same
tolerance as the other reduction tests, twice in a row (the second call runs
on the array the first one left behind).  This file is collected last on
purpose: it must pass in a fresh process and after every other test.
"""
import ctypes

import pytest
import torch

from paper_2211_15634_gb300 import _lib, api

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

NMAX = 4096 * 32768  # capacity stated in include/ps_diffusion3d.h


def seeded(n, dtype, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return (2.0 * torch.rand(n, generator=g, device="cuda", dtype=torch.float64) - 1.0).to(dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [1, 4095, 4097, 1 << 20, NMAX])
def test_dot_static_matches_dot(dtype, n):
    lib = _lib.load()
    code = _lib.PS_F64 if dtype == torch.float64 else _lib.PS_F32
    A, B = seeded(n, dtype, 11), seeded(n, dtype, 12)
    ref = float(api.dot(A, B))
    scale = float(api.dot(A.abs(), B.abs()))
    check_twice(lib, A, B, n, code, ref, scale)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_dot_static_takes_element_aligned_views(dtype):
    """Views that start one element into a buffer (8 or 4 bytes past a 16-byte
    boundary) are accepted: the kernel reads one element at a time."""
    lib = _lib.load()
    code = _lib.PS_F64 if dtype == torch.float64 else _lib.PS_F32
    n = 70001
    A, B = seeded(n + 1, dtype, 21)[1:], seeded(n + 3, dtype, 22)[3:]
    assert A.data_ptr() % 16 != 0 and B.data_ptr() % 16 != 0
    ref = float(api.dot(A.clone(), B.clone()))
    scale = float(api.dot(A.abs(), B.abs()))
    check_twice(lib, A, B, n, code, ref, scale)


def check_twice(lib, A, B, n, code, ref, scale):
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty((), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        st = lib.ps_dot_static(out.data_ptr(), A.data_ptr(), B.data_ptr(), n, code, stream)
        assert st == _lib.PS_OK, lib.ps_last_error()
        torch.cuda.synchronize()
        assert abs(float(out) - ref) <= 1e-13 * scale


def test_dot_static_rejects_sizes_beyond_capacity():
    lib = _lib.load()
    A = seeded(16, torch.float64, 1)
    out = torch.full((), 7.0, dtype=torch.float64, device="cuda")
    st = lib.ps_dot_static(out.data_ptr(), A.data_ptr(), A.data_ptr(), NMAX + 1, _lib.PS_F64,
                           torch.cuda.current_stream().cuda_stream)
    assert st == _lib.PS_ERR_UNSUPPORTED
    assert b"capacity" in lib.ps_last_error()
    torch.cuda.synchronize()
    assert float(out) == 7.0  # nothing was launched
