"""The PyTorch form of the counter-based input generator (inputs.uniform_torch) gives
the numpy form's draws bit for bit - on counters past 2^31, 2^32 and up to 2^64 - 1,
and as whole fields - so that fields too large to generate on the host are the same
fields.  CPU only (the GPU form is checked in tests/test_gpu_fullsize.py)."""
import numpy as np
import torch

from paper_2211_15634_gb300 import inputs


def test_draws_equal_numpy_bit_for_bit():
    idx = np.concatenate([np.arange(0, 4096, dtype=np.uint64),
                          np.array([2**31 - 1, 2**31, 2**32 - 1, 2**32, 2**32 + 5, 2**40 + 17,
                                    2**62, 2**63 - 1, 2**63, 2**64 - 1], dtype=np.uint64)])
    t = torch.from_numpy(idx.view(np.int64))
    for seed in (0, 7, 99, inputs.SEED_CI, inputs.SEED_CI_TRUE, 2**40 + 3, 2**64 - 1):
        assert np.array_equal(inputs.uniform(seed, idx), inputs.uniform_torch(seed, t).numpy())


def test_field_equals_numpy_field():
    nx, ny, nz = 13, 7, 9
    a = inputs.uniform_field(inputs.SEED_CI, nx, ny, nz)
    b = inputs.uniform_field_torch(inputs.SEED_CI, nx, ny, nz, "cpu", planes=2).numpy()
    assert np.array_equal(a, b)
    # the workload's Ci from the torch draws, by the same three operations
    ci = ((torch.from_numpy(b) * 0.5) + 1.0) * (1.0 / inputs.C0)
    assert np.array_equal(inputs.ci_random(nx, ny, nz), ci.numpy())
