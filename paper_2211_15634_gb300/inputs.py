"""Seeded synthetic inputs for the 3-D heat diffusion solver.

This module only *generates* input fields; it holds none of the solver's
arithmetic (no step, no dt, no reduction).  Both the CUDA path and the FP64
reference consume the arrays it returns, so the two always see the same bits.

Fields follow the paper's Fig. 1 set-up (lam=1, c0=2, lx=ly=lz=1,
dx=lx/(nx-1), T=1.7 and Ci=1/c0) with the variable-coefficient workload
layered on top:

* ``Ci = (1/c0) * (1 + 0.5*U)`` with ``U`` uniform in [0, 1) from a
  counter-based splitmix64 stream (one draw per grid point, indexed by the
  point's linear offset);
* ``T0 = 1.7 + exp(-((x-.5)^2 + (y-.5)^2 + (z-.5)^2) / 0.01)`` on the node
  coordinates ``x_i = i*dx`` (both domain ends are nodes);
* "smooth noise": uniform draws on a 9^3 lattice spanning [0,1]^3,
  trilinearly interpolated to the grid nodes (values stay in [0, 1)).

Arrays are C-contiguous with shape ``(nz, ny, nx)`` so the linear offset of
node (i, j, k) is ``i + nx*(j + ny*k)`` (x fastest, as in Julia's
column-major ``T[i,j,k]``).
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Seeds of the standard workloads.
SEED_CI = 2211          # variable Ci of the forward workloads
SEED_CI_TRUE = 15634    # "true" Ci of the inverse problem (smooth noise)
SEED_BATCH_SIZES = 7    # grid sizes of the batched workload
SEED_BATCH_BASE = 1000  # problem p of the batch uses seed 1000 + p

LAM = 1.0
C0 = 2.0
T_BASE = 1.7


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One output of Steele/Lea/Flood's SplitMix64 whose state is ``x``.

    The state is advanced by the golden gamma and then passed through the
    variant-13 finaliser (shifts 30/27/31, multipliers 0xBF58476D1CE4E5B9 and
    0x94D049BB133111EB).  Wrapping uint64 arithmetic throughout.
    """
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64, copy=True)
        z += GOLDEN_GAMMA
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def uniform(seed: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based U[0,1) draws: ``(splitmix64(seed ^ idx*gamma) >> 11) * 2^-53``."""
    with np.errstate(over="ignore"):
        key = np.uint64(seed) ^ (idx.astype(np.uint64) * GOLDEN_GAMMA)
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _as_int64(v: int) -> int:
    """The signed 64-bit integer with the bits of the unsigned 64-bit ``v``."""
    return v - (1 << 64) if v >= (1 << 63) else v


def _shr(z, s: int):
    """Logical right shift by ``s`` of uint64 bit patterns held in an int64 tensor."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def uniform_torch(seed: int, idx):
    """:func:`uniform` for an int64 torch tensor of counters, on any device, bit for bit:
    the same SplitMix64 draw in wrapping int64 arithmetic with logical right shifts
    (for inputs too large to generate on the host)."""
    import torch
    g = _as_int64(int(GOLDEN_GAMMA))
    z = idx.to(torch.int64) * g
    z = z ^ _as_int64(int(seed) & ((1 << 64) - 1))
    z = z + g
    z = z ^ _shr(z, 30)
    z = z * _as_int64(int(_M1))
    z = z ^ _shr(z, 27)
    z = z * _as_int64(int(_M2))
    z = z ^ _shr(z, 31)
    return _shr(z, 11).to(torch.float64) * (2.0 ** -53)


def uniform_field_torch(seed: int, nx: int, ny: int, nz: int, device, planes: int = 32):
    """:func:`uniform_field` generated on ``device`` (float64, shape ``(nz, ny, nx)``),
    ``planes`` z-planes of counters at a time."""
    import torch
    out = torch.empty((nz, ny, nx), dtype=torch.float64, device=device)
    plane = nx * ny
    for k0 in range(0, nz, planes):
        k1 = min(nz, k0 + planes)
        idx = torch.arange(k0 * plane, k1 * plane, dtype=torch.int64, device=device)
        out[k0:k1] = uniform_torch(seed, idx).view(k1 - k0, ny, nx)
    return out


def uniform_field(seed: int, nx: int, ny: int, nz: int, chunk: int = 1 << 24) -> np.ndarray:
    """U[0,1) per node, draw index = linear offset ``i + nx*(j + ny*k)``."""
    n = nx * ny * nz
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = uniform(seed, np.arange(s, e, dtype=np.uint64))
    return out.reshape(nz, ny, nx)


def spacing(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0):
    """Grid spacings ``dd = l_d/(n_d-1)`` (Fig. 1 numerics)."""
    return lx / (nx - 1), ly / (ny - 1), lz / (nz - 1)


def inverse_spacing(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0, lz: float = 1.0):
    """``(_dx, _dy, _dz) = (1/dx, 1/dy, 1/dz)`` as Fig. 1 passes them to the step."""
    dx, dy, dz = spacing(nx, ny, nz, lx, ly, lz)
    return 1.0 / dx, 1.0 / dy, 1.0 / dz


def node_coords(n: int, length: float = 1.0) -> np.ndarray:
    """Node coordinates ``x_i = i*dx``, i = 0..n-1."""
    d = length / (n - 1)
    return np.arange(n, dtype=np.float64) * d


def ci_random(nx: int, ny: int, nz: int, seed: int = SEED_CI, c0: float = C0) -> np.ndarray:
    """``Ci = (1/c0) * (1 + 0.5*U[0,1))`` from the seeded counter stream."""
    u = uniform_field(seed, nx, ny, nz)
    u *= 0.5
    u += 1.0
    u *= 1.0 / c0
    return u


def ci_constant(nx: int, ny: int, nz: int, c0: float = C0) -> np.ndarray:
    """The paper's own ``Ci = ones/c0``."""
    return np.full((nz, ny, nx), 1.0 / c0)


def t0_gaussian(nx: int, ny: int, nz: int, base: float = T_BASE, width: float = 0.01) -> np.ndarray:
    """``T0 = base + exp(-((x-.5)^2 + (y-.5)^2 + (z-.5)^2)/width)`` on the nodes."""
    x = (node_coords(nx) - 0.5) ** 2
    y = (node_coords(ny) - 0.5) ** 2
    z = (node_coords(nz) - 0.5) ** 2
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for k in range(nz):
        r2 = (x[None, :] + y[:, None]) + z[k]
        np.exp(-r2 / width, out=out[k])
    out += base
    return out


def t0_constant(nx: int, ny: int, nz: int, value: float = T_BASE) -> np.ndarray:
    """The paper's own ``T = ones*1.7``."""
    return np.full((nz, ny, nx), value)


def smooth_noise(nx: int, ny: int, nz: int, seed: int, lattice: int = 9) -> np.ndarray:
    """U[0,1) on a ``lattice^3`` grid spanning [0,1]^3, trilinearly interpolated."""
    m = lattice
    coarse = uniform_field(seed, m, m, m)  # (m, m, m), index [k, j, i]

    def axis(n):
        t = node_coords(n) * (m - 1)
        i0 = np.minimum(np.floor(t).astype(np.int64), m - 2)
        f = t - i0
        return i0, f

    ix, fx = axis(nx)
    iy, fy = axis(ny)
    iz, fz = axis(nz)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for k in range(nz):
        acc = np.zeros((ny, nx))
        for dk, wk in ((0, 1.0 - fz[k]), (1, fz[k])):
            plane = coarse[iz[k] + dk]
            for dj in (0, 1):
                wj = (1.0 - fy) if dj == 0 else fy
                rows = plane[iy + dj]  # (ny, m)
                for di in (0, 1):
                    wi = (1.0 - fx) if di == 0 else fx
                    acc += wk * wj[:, None] * wi[None, :] * rows[:, ix + di]
        out[k] = acc
    return out


def ci_smooth(nx: int, ny: int, nz: int, seed: int = SEED_CI_TRUE, c0: float = C0) -> np.ndarray:
    """True Ci of the inverse problem: ``(1/c0) * (1 + 0.5*smooth_noise)``."""
    s = smooth_noise(nx, ny, nz, seed)
    return (1.0 / c0) * (1.0 + 0.5 * s)


def batch_sizes(nprob: int, lo: int = 32, hi: int = 160, seed: int = SEED_BATCH_SIZES) -> np.ndarray:
    """Cubic grid sizes n_p uniform on the integers {lo..hi}."""
    u = uniform(seed, np.arange(nprob, dtype=np.uint64))
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def batch_problem(p: int, n: int, c0: float = C0):
    """Inputs of problem p of the batch: (T0, Ci) on an n^3 grid, Ci seeded 1000+p."""
    return t0_gaussian(n, n, n), ci_random(n, n, n, seed=SEED_BATCH_BASE + p, c0=c0)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Generic U[lo,hi) field (test vectors for dot-product and FD checks)."""
    n = int(np.prod(shape))
    u = uniform(seed, np.arange(n, dtype=np.uint64))
    return (lo + (hi - lo) * u).reshape(shape)
