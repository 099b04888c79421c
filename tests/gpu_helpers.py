"""Shared helpers of the GPU parity tests (test code, not product)."""
import numpy as np
import torch

from paper_2211_15634_gb300 import inputs


def to_dev(a: np.ndarray, dtype=torch.float64) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu", torch.float64).numpy()


def rel_linf(a, b) -> float:
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def problem(nx, ny, nz, seed=inputs.SEED_CI, lam=1.0, gaussian=True):
    """Workload-shaped fields: Gaussian T0 (or random), seeded random Ci, Fig. 1 dt."""
    Ci = inputs.ci_random(nx, ny, nz, seed=seed)
    T0 = inputs.t0_gaussian(nx, ny, nz) if gaussian else \
        1.7 + inputs.random_field((nz, ny, nx), seed + 99, 0.0, 1.0)
    dx, dy, dz = inputs.spacing(nx, ny, nz)
    dt = min(dx * dx, dy * dy, dz * dz) / lam / Ci.max() / 6.1
    return T0, Ci, lam, dt, inputs.inverse_spacing(nx, ny, nz)


def light_cone_reference(oracle, T0, Ci, lam, dt, inv, nt, points):
    """Oracle values of T(nt) at `points` [(i, j, k)], each from the sub-block of
    half-width nt around it (clipped at the domain): the node's value after nt
    steps depends on nothing outside that block, and a face of the block that is
    not a domain face is nt nodes away, so its (wrongly fixed) values cannot
    reach the node within nt steps."""
    nz, ny, nx = T0.shape
    out = []
    for (i, j, k) in points:
        i0, i1 = max(0, i - nt), min(nx, i + nt + 1)
        j0, j1 = max(0, j - nt), min(ny, j + nt + 1)
        k0, k1 = max(0, k - nt), min(nz, k + nt + 1)
        sub_T = np.ascontiguousarray(T0[k0:k1, j0:j1, i0:i1])
        sub_C = np.ascontiguousarray(Ci[k0:k1, j0:j1, i0:i1])
        if min(sub_T.shape) < 3:
            out.append(T0[k, j, i])  # a boundary node never changes
            continue
        res = oracle.run(sub_T, sub_C, lam, dt, *inv, nt)
        out.append(res[k - k0, j - j0, i - i0])
    return np.array(out)
