"""The eager PyTorch comparison solver that bench.py times beside the library (Fig. 1's
step as whole-field slice expressions, the analogue of the paper's array-broadcast
comparison) computes the same thing as the FP64 oracle: a wrong comparison program
would otherwise still give a number."""
import pytest
import torch

import bench
import oracle
from gpu_helpers import problem, rel_linf, to_dev, to_host

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("nt", [1, 9])
def test_eager_solver_matches_oracle(nt):
    nx, ny, nz = 37, 29, 23
    T0, Ci, lam, dt, inv = problem(nx, ny, nz, gaussian=False)
    T = to_dev(T0)
    T2 = T.clone()
    out = bench.torch_eager_run(T, T2, to_dev(Ci), lam, dt, inv, nt)
    ref = oracle.run(T0, Ci, lam, dt, *inv, nt)
    assert rel_linf(to_host(out), ref) <= 1e-12
