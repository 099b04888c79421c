#!/usr/bin/env python
"""Benchmark: 3-D diffusion T_eff at 512^3 FP64, nt = 100 (Fig. 1 workload).

One "step" is one pass of the hot path over one synthetic input: the stable
dt from maximum(Ci) reduced on the GPU, then the Fig. 1 time loop (boundary
copy and nt steps with swapped buffers).  T_eff = 3 * nx*ny*nz * 8 bytes *
nt / time (read T and Ci, write T2 per step).  Inputs (3 x 1 GiB) are larger
than the 129 MB L2, so no flush is needed between iterations.

Prints one JSON line on rank 0.  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (bounded samples of the same workload).
Multi-GPU (torchrun): every rank runs an independent replica.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-D diffusion T_eff GB/s (% HBM peak) FP64/FP32 at 512^3; gradient/forward time"
PAPER_TEFF_A100 = 1262.0  # GB/s, FP64 512^3 on an A100 SXM4 (Sect. Results); another machine
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=512)
    p.add_argument("--nt", type=int, default=100)
    p.add_argument("--no-secondary", action="store_true", help="skip FP32 / gradient / batch lines")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=0,
                   help="problems timed end to end (0: --steps, the device-timed step count)")
    p.add_argument("--kernel-loop", choices=["step", "adjoint", "adjoint2", "batch", "step2d", "states"],
                   default=None,
                   help="profiling aid: launch only this kernel --reps times at --size (no JSON); "
                        "step2d on a --size^2 grid; states: the FP32 state-keeping loop of --reps "
                        "states in fused pairs that keep both states")
    p.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    p.add_argument("--field", choices=["gauss", "sine", "gauss_dev"], default="gauss",
                   help="kernel loop step (FP64): the workload's Gaussian on 1.7, or a field that leaves "
                        "one binade (see general_path_fields)")
    p.add_argument("--reps", type=int, default=4)
    p.add_argument("--batch-count", type=int, default=256,
                   help="kernel loop batch: the first this many problems of the 256-problem workload")
    p.add_argument("--comp", action="store_true",
                   help="kernel loop step (FP32): the compensated step on the two-float state")
    p.add_argument("--temporal2", action="store_true",
                   help="kernel loop step: fused step pairs (each rep is two two-step passes)")
    p.add_argument("--plain-ci", action="store_true",
                   help="kernel loop: FP64 step/adjoint/batch on Ci as given instead of the pre-scaled field")
    p.add_argument("--zslab", action="store_true",
                   help="one problem of 512 x 512 x (510 N + 2) nodes split into z-slabs over the N "
                        "ranks (each rank 512^3 with its halos), halo exchange per step (NCCL)")
    p.add_argument("--batch-kernel", choices=["zmarch", "column"], default="zmarch",
                   help="kernel loop batch: the TMA z-march on padded rows, or the column march")
    return p.parse_args()


def run_kernel_loop(args):
    """Launch one kernel family a few times on --size^3 workload fields (for ncu)."""
    import torch
    from paper_2211_15634_gb300 import api, inputs
    if args.kernel_loop == "batch":
        return run_batch_loop(args)
    if args.kernel_loop == "step2d":
        return run_step2d_loop(args)
    n = args.size
    T0, Ci, inv = fields(n)
    dev = torch.device("cuda")
    T = torch.from_numpy(T0).to(dev)
    C = torch.from_numpy(Ci).to(dev)
    if args.field != "gauss":
        T = dict(general_path_fields(torch, n, dev))[args.field]
    if args.dtype == "f32":
        T, C = api.to_deviation(T, 1.7), api.to_f32(C)
    T2 = T.clone()
    dt = api.stable_dt(C, 1.0)
    if args.kernel_loop == "step":
        # FP64: the pre-scaled coefficient of the headline step (--plain-ci: Ci as given)
        scaled = args.dtype == "f64" and not args.plain_ci
        Cs = api.scale_ci(C, 1.0, dt, inv) if scaled else C
        comp = api.compensation_fields(T) if (args.comp and args.dtype == "f32") else None
        for i in range(args.reps):
            src, dst = (T, T2) if i % 2 == 0 else (T2, T)
            if comp is not None:
                api.step_compensated(dst, src, comp[(i + 1) % 2], comp[i % 2], Cs, 1.0, dt, inv)
                continue
            if args.temporal2:  # two fused two-step passes (plus the boundary copy); nt = 4
                # keeps the result in `src`, as an even step count must
                api.run(src, dst, Cs, 1.0, dt, inv, 4, ci_scaled=scaled, temporal2=True)
            else:
                api.step(dst, src, Cs, 1.0, dt, inv, ci_scaled=scaled)
        name = "compensated FP32 step" if comp is not None else api.step_kernel_name(
            T2, T, Cs, 1.0, dt, inv, ci_scaled=scaled, temporal2=args.temporal2)
    elif args.kernel_loop == "states":
        # FP32: --reps states kept, in fused pairs that write both states
        if args.dtype != "f32":
            raise SystemExit("--kernel-loop states is FP32 (--dtype f32)")
        block = api.StateBlock(T, args.reps, boundary=False)
        api.run_states(T, block, 1, C, 1.0, dt, inv, args.reps, temporal2=True)
        name = "state-keeping loop (fused pairs keeping both states)"
    elif args.kernel_loop == "adjoint2":
        # FP32: two transposed steps per pass (states T and T2)
        if args.dtype != "f32":
            raise SystemExit("--kernel-loop adjoint2 is FP32 (--dtype f32)")
        ybar = T2 - T.mean()
        Tbar = torch.empty_like(T)
        Cib = torch.zeros_like(T)
        S0 = T.clone()
        for _ in range(args.reps):
            api.adjoint2(Tbar, Cib, ybar, T, S0, C, 1.0, dt, inv)
        name = "adjoint2 (fused pair)"
    else:
        # FP64: the transposed step on the pre-scaled coefficient (--plain-ci: on Ci)
        scaled = args.dtype == "f64" and not args.plain_ci
        Cs = api.scale_ci(C, 1.0, dt, inv) if scaled else C
        ybar = T2 - T.mean()
        Tbar = torch.empty_like(T)
        Cib = torch.zeros_like(T)
        for _ in range(args.reps):
            api.adjoint(Tbar, Cib, ybar, T, Cs, 1.0, dt, inv, ci_scaled=scaled)
        name = "adjoint (pre-scaled)" if scaled else "adjoint"
    torch.cuda.synchronize()
    log(f"kernel loop done: {name} x{args.reps} at {n}^3 {args.dtype}, device_error={api.device_error()}")
    return 0


def fields2d(torch, api, inputs, n2, dtype, dev):
    """The 2-D workload on an n2 x n2 grid: a Gaussian T on 1.7, random Ci, dt from
    maximum(Ci); FP64 on the pre-scaled coefficient, FP32 in deviation storage.
    Returns (T, C, dt, inverse spacings, ci_scaled)."""
    x = torch.arange(n2, device=dev, dtype=torch.float64) / (n2 - 1)
    T2d = (1.7 + torch.exp(-((x[None, :] - 0.5) ** 2 + (x[:, None] - 0.5) ** 2) / 0.01)).contiguous()
    C2d = torch.from_numpy(inputs.ci_random(n2, n2, 1)[0]).to(dev)
    if dtype == torch.float32:
        T2d, C2d = api.to_deviation(T2d, 1.7), api.to_f32(C2d)
    dt2 = api.stable_dt2d(C2d)
    inv2 = (float(n2 - 1), float(n2 - 1))
    scaled2 = dtype == torch.float64
    if scaled2:
        C2d = api.scale_ci(C2d, 1.0, dt2, inv2)
    return T2d, C2d, dt2, inv2, scaled2


def run_step2d_loop(args):
    """Launch the 2-D step --reps times on the --size^2 workload (for ncu)."""
    import torch
    from paper_2211_15634_gb300 import api, inputs
    dev = torch.device("cuda")
    dtype = torch.float64 if args.dtype == "f64" else torch.float32
    T, C, dt, inv, scaled = fields2d(torch, api, inputs, args.size, dtype, dev)
    T2 = T.clone()
    for i in range(args.reps):
        src, dst = (T, T2) if i % 2 == 0 else (T2, T)
        api.step2d(dst, src, C, 1.0, dt, inv, ci_scaled=scaled)
    torch.cuda.synchronize()
    log(f"kernel loop done: step2d x{args.reps} at {args.size}^2 {args.dtype}, "
        f"device_error={api.device_error()}")
    return 0


def batch_workload(torch, api, inputs, dtype, dev, count=256, pitched=False, ci_scaled=False):
    """The batched workload: problem q is an n_q^3 grid, n_q uniform in 32..160.

    ``pitched``: fields with rows padded to 16 bytes (the z-march batch's layout);
    ``ci_scaled`` (FP64): each Ci field holds the pre-scaled dt*lam*_dx^2*Ci.
    Returns the problems and the algorithmic bytes of one step (3 n^3 per problem)."""
    probs, nbytes = [], 0
    esz = 8 if dtype == torch.float64 else 4
    for q, nq in enumerate(inputs.batch_sizes(256)[:count]):
        nq = int(nq)
        T0q, Ciq = inputs.batch_problem(q, nq)
        Tq = torch.from_numpy(T0q).to(dev)
        Cq = torch.from_numpy(Ciq).to(dev)
        if dtype == torch.float32:
            Tq = api.to_deviation(Tq, 1.7)
            Cq = api.to_f32(Cq)
        dtq = api.stable_dt(Cq, 1.0)
        inv = inputs.inverse_spacing(nq, nq, nq)
        if ci_scaled:
            Cq = api.scale_ci(Cq, 1.0, dtq, inv)
        if pitched:
            Tq, Cq = api.pitched_copy(Tq), api.pitched_copy(Cq)
        T2q = api.pitched_copy(Tq) if pitched else Tq.clone()
        probs.append(dict(T=Tq, T2=T2q, Ci=Cq, lam=1.0, dt=dtq, inv_spacing=inv))
        nbytes += 3 * nq ** 3 * esz
    return probs, nbytes


def run_batch_loop(args):
    import torch
    from paper_2211_15634_gb300 import api, inputs
    dtype = torch.float64 if args.dtype == "f64" else torch.float32
    zm = args.batch_kernel == "zmarch"
    scaled = zm and dtype == torch.float64 and not args.plain_ci
    probs, nbytes = batch_workload(torch, api, inputs, dtype, torch.device("cuda"), args.batch_count,
                                   pitched=zm, ci_scaled=scaled)
    b = api.Batch(probs, kernel=args.batch_kernel, ci_scaled=scaled)
    for it in range(args.reps):
        b.step(it & 1)
    torch.cuda.synchronize()
    name = "k_batch_zmarch" if zm else "k_batch_step"
    log(f"kernel loop done: {name} x{args.reps}, {len(probs)} problems, {b.nitems} items, "
        f"{nbytes / 1e9:.2f} GB per step, {args.dtype}{' pre-scaled' if scaled else ''}, "
        f"device_error={api.device_error()}")
    return 0


# ------------------------------------------------------------------ system
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def median_ci95(xs):
    """Median and a distribution-free 95% confidence interval of the median (order
    statistics of the binomial(n, 1/2) law)."""
    xs = sorted(xs)
    n = len(xs)
    if n < 6:
        return statistics.median(xs), xs[0], xs[-1]
    # largest j with P(Bin(n, 1/2) <= j-1) <= 0.025: the interval is [x_(j), x_(n-j+1)]
    cdf, j = 0.0, 0
    for k in range(n + 1):
        cdf += math.comb(n, k) / 2.0 ** n
        if cdf > 0.025:
            j = k
            break
    j = max(j, 1)
    return statistics.median(xs), xs[j - 1], xs[n - j]


def step_samples(step_ms, bytes_per_step):
    """Per-step device times (CUDA events around each step) as T_eff samples."""
    med, lo, hi = median_ci95(step_ms)
    rate = lambda ms: round(bytes_per_step / (ms / 1e3) / 1e9, 1)  # noqa: E731
    return {"n": len(step_ms), "median_ms": round(med, 3), "ci95_ms": [round(lo, 3), round(hi, 3)],
            "median_gbs": rate(med), "ci95_gbs": [rate(hi), rate(lo)]}


def max_over_ranks(seconds: float, device=None) -> float:
    """Slowest rank's time (all ranks get it); the local value without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, slowest_seconds: float, world: int) -> float:
    """Units processed by all ranks (replicas: each does units_per_rank) per second."""
    return world * units_per_rank / slowest_seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum clock and the throttle reasons seen Active in
        nvidia-smi CSV lines of FIELDS (malformed lines skipped); None without samples."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def source_digest(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, digest: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged.

    Lines: ``TRAFFIC <kernel> <n> <bytes_per_launch> <source digest>``.
    """
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        f = ln.split()
        if len(f) == 5 and f[0] == "TRAFFIC" and f[1] == kernel and f[4] == digest:
            return float(f[3]) * (n ** 3) / (int(f[2]) ** 3)
    return None


# --------------------------------------------------------------- workloads
def fields(n):
    from paper_2211_15634_gb300 import inputs
    T0 = inputs.t0_gaussian(n, n, n)
    Ci = inputs.ci_random(n, n, n)
    return T0, Ci, inputs.inverse_spacing(n, n, n)


def big_fields(n, dtype, dev):
    """Workload fields of an n^3 grid built plane by plane on the host (bounded
    host memory), uploaded as `dtype`; FP32 temperatures as deviations from 1.7."""
    import torch
    from paper_2211_15634_gb300 import inputs
    T = torch.empty((n, n, n), dtype=dtype, device=dev)
    C = torch.empty((n, n, n), dtype=dtype, device=dev)
    x = (inputs.node_coords(n) - 0.5) ** 2
    plane = n * n
    for k in range(n):
        t = np.exp(-((x[None, :] + x[:, None]) + x[k]) / 0.01)
        if dtype == torch.float64:
            t = t + 1.7
        idx = np.arange(k * plane, (k + 1) * plane, dtype=np.uint64)
        c = (1.0 / inputs.C0) * (1.0 + 0.5 * inputs.uniform(inputs.SEED_CI, idx)).reshape(n, n)
        T[k].copy_(torch.from_numpy(t))
        C[k].copy_(torch.from_numpy(c))
    return T, C


def oracle_sample(T0, Ci, inv, steps, threads):
    """Time the FP64 oracle for `steps` steps on the whole field (host cores)."""
    import oracle
    n = T0.shape[0]
    oracle.set_threads(threads)
    dx = 1.0 / (n - 1)
    dt = oracle.stable_dt(dx, dx, dx, 1.0, oracle.maximum(Ci))
    t = time.perf_counter()
    oracle.run(T0, Ci, 1.0, dt, *inv, steps)
    el = time.perf_counter() - t
    return el


def oracle_rate(T0, Ci, inv, threads, budget_s):
    """(T_eff GB/s, steps, seconds) of the FP64 oracle on `threads` host threads, for about
    budget_s seconds of steps (one probe step sizes the sample)."""
    n = T0.shape[0]
    t1 = oracle_sample(T0, Ci, inv, 1, threads)
    steps = int(max(1, min(100, budget_s / max(t1, 1e-3))))
    el = oracle_sample(T0, Ci, inv, steps, threads)
    return 3 * n ** 3 * 8 * steps / el / 1e9, steps, el


def cpu_baseline(T0, Ci, inv, budget_s=15.0):
    """The oracle on all host cores (OpenMP over z) on the benchmark's fields; beside it the
    serial oracle on the same fields and both on the 256^3 fields (a few seconds each)."""
    import oracle
    threads = max(1, oracle.max_threads())
    n = T0.shape[0]
    gbs, steps, el = oracle_rate(T0, Ci, inv, threads, budget_s)
    serial, s_steps, _ = oracle_rate(T0, Ci, inv, 1, 5.0)
    T0s, Cis, invs = fields(256)
    omp256, _, _ = oracle_rate(T0s, Cis, invs, threads, 2.0)
    serial256, _, _ = oracle_rate(T0s, Cis, invs, 1, 3.0)
    oracle.set_threads(1)
    return {"value": round(gbs, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps (plus the initial copy) on the full {n}^3 fields, "
                      f"{el:.1f} s on {threads} host threads",
            "serial_value": round(serial, 3),
            "serial_sample": f"{s_steps} steps on the same fields, 1 thread",
            "at_256": {"value": round(omp256, 3), "serial_value": round(serial256, 3)}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n = args.size
    T0, Ci, inv = fields(n)
    threads = max(1, oracle.max_threads())
    t1 = oracle_sample(T0, Ci, inv, 1, threads)
    total = args.steps + args.warmup
    steps = int(max(1, min(args.nt, 150.0 / total / max(t1, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample(T0, Ci, inv, steps, threads)
    times = [oracle_sample(T0, Ci, inv, steps, threads) for _ in range(args.steps)]
    el = sum(times)
    gbs = 3 * n ** 3 * 8 * steps * args.steps / el / 1e9
    line = {
        "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": f"diffusion3d FP64 {n}^3 Gaussian T0, random Ci, nt={args.nt}",
                   "nx": n, "ny": n, "nz": n, "nt": args.nt, "parallelism": "host threads"},
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step = {steps} oracle time steps on the full {n}^3 fields"},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- our path
def torch_eager_step(Ta, Tb, C, lam, dt, inv):
    """Fig. 1's step! written as whole-field PyTorch slice expressions on (nz, ny, nx)
    tensors (one kernel per operation): the analogue of the paper's GPU array-broadcast
    comparison solver.  Writes Tb's interior from Ta; Tb's boundary is left as it is.
    Same association order as Fig. 1: T + dt*(lam*Ci*((d2x*_dx^2 + d2y*_dy^2) + d2z*_dz^2))."""
    ax, ay, az = (v * v for v in inv)
    c = Ta[1:-1, 1:-1, 1:-1]
    d2x = (Ta[1:-1, 1:-1, 2:] - c) - (c - Ta[1:-1, 1:-1, :-2])
    d2y = (Ta[1:-1, 2:, 1:-1] - c) - (c - Ta[1:-1, :-2, 1:-1])
    d2z = (Ta[2:, 1:-1, 1:-1] - c) - (c - Ta[:-2, 1:-1, 1:-1])
    Tb[1:-1, 1:-1, 1:-1] = c + dt * (lam * C[1:-1, 1:-1, 1:-1] * ((d2x * ax + d2y * ay) + d2z * az))


def torch_eager_run(T, T2, C, lam, dt, inv, nt):
    """nt eager steps with the buffers swapped (T2's boundary must equal T's); returns
    the tensor holding T(nt)."""
    for it in range(nt):
        if it % 2 == 0:
            torch_eager_step(T, T2, C, lam, dt, inv)
        else:
            torch_eager_step(T2, T, C, lam, dt, inv)
    return T2 if nt % 2 else T


def torch_eager_teff(torch, T, T2, C, dt, inv, timed, nt=10):
    """T_eff of the eager slice-expression solver on the same fields, by the same
    3-array count (checked against the oracle in the GPU tests)."""
    n = T.shape[0]
    t = timed(lambda: torch_eager_run(T, T2, C, 1.0, dt, inv, nt), reps=2)
    return round(3 * n ** 3 * T.element_size() * nt / t / 1e9, 1)


def general_path_warp_fraction(torch, T):
    """Share of the warp-planes of the pre-scaled FP64 step (k_zmarch<F64_SCALED4>: a warp
    owns 128 consecutive nodes of a row, four per lane) in which some lane's stencil
    values do not all share the sign and exponent of its first centre, so that the
    warp takes the general fixed-point path - on the field T as given (a host-side
    count over the field, not a device counter; nodes at the x edges are counted like
    the others)."""
    n = T.shape[2]
    H = ((T.view(torch.int64) >> 52) & 0xFFF).to(torch.int16)
    L = n // 4
    A = H[1:-1, 1:-1, :].reshape(n - 2, n - 2, L, 4)
    ref = A[..., 0]
    f = (A == ref[..., None]).all(-1)
    for nb in (H[1:-1, :-2, :], H[1:-1, 2:, :], H[:-2, 1:-1, :], H[2:, 1:-1, :]):
        f &= (nb.reshape(n - 2, n - 2, L, 4) == ref[..., None]).all(-1)
    f[..., 1:] &= A[..., :-1, 3] == ref[..., 1:]
    f[..., :-1] &= A[..., 1:, 0] == ref[..., :-1]
    pad = (-L) % 32  # lanes past the grid's last tile compute nothing
    if pad:
        f = torch.cat([f, torch.ones(n - 2, n - 2, pad, dtype=torch.bool, device=f.device)], dim=-1)
    warp_fast = f.reshape(n - 2, n - 2, (L + pad) // 32, 32).all(-1)
    return round(1.0 - float(warp_fast.float().mean()), 4)


def general_path_fields(torch, n, dev):
    """Fields on which the FP64 step leaves the one-binade fast path: the sine mode
    shifted to cross zero, sin(pi x) sin(pi y) sin(pi z) - 1/2 (signs and many binades
    near its zero set), and the Gaussian stored as its deviation from 1.7 in FP64
    (exp(-r^2/0.01): positive, but a new binade every few nodes in its tails)."""
    from paper_2211_15634_gb300 import inputs
    x = torch.from_numpy(inputs.node_coords(n)).to(dev)
    s = torch.sin(torch.pi * x)
    yield "sine", (s[:, None, None] * s[None, :, None] * s[None, None, :] - 0.5).contiguous()
    d = (x - 0.5) ** 2
    yield "gauss_dev", torch.exp(-((d[:, None, None] + d[None, :, None]) + d[None, None, :]) / 0.01).contiguous()


def secondary_metrics(torch, api, ag, inputs, log):
    """FP32 512^3, gradient/forward ratio at 256^3, batched workload."""
    out = {}
    dev = torch.device("cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = ev(), ev()
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        return statistics.median(ts)

    # FP32 deviation storage at 512^3, plain and compensated
    n, nt = 512, 100
    T0, Ci, inv = fields(n)
    T = torch.from_numpy(T0).to(dev)
    C = torch.from_numpy(Ci).to(dev)
    # FP64 on Ci as given (three-term emulated step, no pre-scaled coefficient)
    T2 = T.clone()
    dt = api.stable_dt(C, 1.0)
    t = timed(lambda: api.run(T, T2, C, 1.0, dt, inv, nt, graph=True))
    out["fp64_512_plain_ci_teff_gbs"] = round(3 * n ** 3 * 8 * nt / t / 1e9, 1)
    # FP64 in fused step pairs (temporal blocking of depth 2) on the pre-scaled coefficient
    Cs = api.scale_ci(C, 1.0, dt, inv)
    t = timed(lambda: api.run(T, T2, Cs, 1.0, dt, inv, nt, graph=True, ci_scaled=True, temporal2=True))
    out["fp64_512_temporal2_teff_gbs"] = round(3 * n ** 3 * 8 * nt / t / 1e9, 1)
    # the same step as plain PyTorch tensor expressions (slices of the whole field)
    out["fp64_512_torch_eager_teff_gbs"] = torch_eager_teff(torch, T, T2, C, dt, inv, timed)
    # the headline field's share of warps on the general path, then the same pre-scaled
    # step on fields that leave one binade (general fixed-point path)
    out["fp64_512_gauss_general_warp_fraction"] = general_path_warp_fraction(torch, T)
    for name, Tg in general_path_fields(torch, n, dev):
        out[f"fp64_512_{name}_general_warp_fraction"] = general_path_warp_fraction(torch, Tg)
        T2.copy_(Tg)
        t = timed(lambda: api.run(Tg, T2, Cs, 1.0, dt, inv, nt, graph=True, ci_scaled=True))
        out[f"fp64_512_{name}_teff_gbs"] = round(3 * n ** 3 * 8 * nt / t / 1e9, 1)
        del Tg
        api.clear_graph_cache()
    del T2, Cs
    api.clear_graph_cache()
    D = api.to_deviation(T, 1.7)
    C32 = api.to_f32(C)
    del T, C
    D2 = D.clone()
    comp = api.compensation_fields(D)
    dt = api.stable_dt(C32, 1.0)
    t = timed(lambda: api.run(D, D2, C32, 1.0, dt, inv, nt, graph=True))
    out["fp32_512_teff_gbs"] = round(3 * n ** 3 * 4 * nt / t / 1e9, 1)
    t = timed(lambda: api.run(D, D2, C32, 1.0, dt, inv, nt, comp=comp, graph=True))
    out["fp32c_512_teff_gbs"] = round(5 * n ** 3 * 4 * nt / t / 1e9, 1)
    # fused step pairs: HBM traffic of one step per two (T_eff may exceed the copy rate)
    t = timed(lambda: api.run(D, D2, C32, 1.0, dt, inv, nt, graph=True, temporal2=True))
    out["fp32_512_temporal2_teff_gbs"] = round(3 * n ** 3 * 4 * nt / t / 1e9, 1)
    del D, D2, comp, C32
    api.clear_graph_cache()
    torch.cuda.empty_cache()

    # size checks: FP64 768^3 and FP32 1024^3 (nt = 100)
    for name, n, dtype in (("fp64_768", 768, torch.float64), ("fp32_1024", 1024, torch.float32)):
        nt = 100
        T, C = big_fields(n, dtype, dev)
        T2 = T.clone()
        dt = api.stable_dt(C, 1.0)
        inv = inputs.inverse_spacing(n, n, n)
        scaled = dtype == torch.float64
        if scaled:
            api.scale_ci(C, 1.0, dt, inv, out=C)
        t = timed(lambda: api.run(T, T2, C, 1.0, dt, inv, nt, graph=True, ci_scaled=scaled), reps=2)
        esz = 8 if dtype == torch.float64 else 4
        out[f"{name}_teff_gbs"] = round(3 * n ** 3 * esz * nt / t / 1e9, 1)
        if not scaled:
            t = timed(lambda: api.run(T, T2, C, 1.0, dt, inv, nt, graph=True, temporal2=True), reps=2)
            out[f"{name}_temporal2_teff_gbs"] = round(3 * n ** 3 * esz * nt / t / 1e9, 1)
        del T, T2, C
        api.clear_graph_cache()
        torch.cuda.empty_cache()

    # FP32 error against the FP64 oracle at 256^3 (nt = 100 and 1000), plain and compensated
    # (two-float state started from the two-float deviation of T0), each split in two:
    #   arithmetic: the oracle run on exactly the state the GPU starts from (D0, or D0 + E0,
    #               in FP64) and on the FP32-rounded Ci - the step's own roundings only;
    #   storage:    the oracle run on the FP64 T0 and Ci - rounding the inputs counts too.
    import oracle
    n = 256
    T0, Ci, inv = fields(n)
    dt = oracle.stable_dt(1.0 / (n - 1), 1.0 / (n - 1), 1.0 / (n - 1), 1.0, oracle.maximum(Ci))
    oracle.set_threads(max(1, oracle.max_threads()))
    Td = torch.from_numpy(T0).to(dev)
    C32 = api.to_f32(torch.from_numpy(Ci).to(dev))
    Ci32 = C32.double().cpu().numpy()
    D0p = api.to_deviation(Td, 1.7)
    D0c, E0c = api.to_deviation_pair(Td, 1.7)
    start_plain = D0p.double().cpu().numpy()
    start_comp = api.from_deviation_pair(D0c, E0c, 0.0).cpu().numpy()
    for nt in (100, 1000):
        ref_store = oracle.run(T0, Ci, 1.0, dt, *inv, nt)
        scale = float(np.max(np.abs(ref_store)))
        for tag, comp in (("fp32", False), ("fp32c", True)):
            if comp:
                D = D0c.clone()
                cbuf = api.compensation_fields(D, E0c)
                res = api.run(D, torch.empty_like(D), C32, 1.0, dt, inv, nt, comp=cbuf)
                got = api.from_deviation_pair(res, cbuf[nt % 2], 1.7).cpu().numpy()
                ref_arith = oracle.run(start_comp, Ci32, 1.0, dt, *inv, nt) + 1.7
            else:
                D = D0p.clone()
                res = api.run(D, torch.empty_like(D), C32, 1.0, dt, inv, nt)
                got = api.from_deviation(res, 1.7).cpu().numpy()
                ref_arith = oracle.run(start_plain, Ci32, 1.0, dt, *inv, nt) + 1.7
            out[f"{tag}_relerr_256_nt{nt}"] = float(f"{np.max(np.abs(got - ref_store)) / scale:.3e}")
            out[f"{tag}_arith_relerr_256_nt{nt}"] = float(f"{np.max(np.abs(got - ref_arith)) / scale:.3e}")
        C64 = torch.from_numpy(Ci).to(dev)
        for tag, scaled in (("fp64", True), ("fp64_plain_ci", False)):
            T64, T64b = Td.clone(), Td.clone()
            Cx = api.scale_ci(C64, 1.0, dt, inv) if scaled else C64
            got = api.run(T64, T64b, Cx, 1.0, dt, inv, nt, ci_scaled=scaled).cpu().numpy()
            out[f"{tag}_relerr_256_nt{nt}"] = float(f"{np.max(np.abs(got - ref_store)) / scale:.3e}")
    oracle.set_threads(1)
    del Td, C32, D, D0p, D0c, E0c
    torch.cuda.empty_cache()

    # gradient / forward at 256^3, nt = 200: L = 1/2||T(nt) - T_obs||^2, dL/dCi and dL/dT0.
    # The forward run it is compared with is the library's default time loop of the same
    # problem (graph-captured one-step launches; FP64 on the pre-scaled coefficient, as the
    # gradient's own forward); FP32 also against the fused-pair forward (grad_over_fwd2),
    # its fastest.  Checkpoints every ceil(sqrt(nt)) steps (recompute per segment), and
    # every state kept (27 GB at 256^3 FP64, no recompute).
    n, nt = 256, 200
    T0 = inputs.t0_gaussian(n, n, n)
    Ct = inputs.ci_smooth(n, n, n)
    inv = inputs.inverse_spacing(n, n, n)
    dx = 1.0 / (n - 1)
    dt = dx * dx / 1.0 / (1.5 / inputs.C0) / 6.1
    for name, dtype in (("fp64", torch.float64), ("fp32", torch.float32)):
        if dtype == torch.float64:
            Td = torch.from_numpy(T0).to(dev)
            Ctd = torch.from_numpy(Ct).to(dev)
            Cd = torch.full_like(Td, 1.0 / inputs.C0)
        else:
            Td = api.to_deviation(torch.from_numpy(T0).to(dev), 1.7)
            Ctd = api.to_f32(torch.from_numpy(Ct).to(dev))
            Cd = torch.full_like(Td, 1.0 / inputs.C0)
        a, b = Td.clone(), Td.clone()
        Tobs = api.run(a, b, Ctd, 1.0, dt, inv, nt).clone()
        fa, fb = Td.clone(), Td.clone()
        Cf, scaled = ag.coefficient(Cd, 1.0, dt, inv)
        t_fwd = timed(lambda: api.run(fa, fb, Cf, 1.0, dt, inv, nt, graph=True, ci_scaled=scaled))
        out[f"fwd_256_{name}_ms"] = round(1e3 * t_fwd, 2)
        t_fwd2 = None
        if dtype == torch.float32:
            t_fwd2 = timed(lambda: api.run(fa, fb, Cf, 1.0, dt, inv, nt, graph=True, temporal2=True))
            out[f"fwd2_256_{name}_ms"] = round(1e3 * t_fwd2, 2)
        # the transposed step alone (CUDA events, warm), before the gradient runs: releasing
        # their 13-27 GB state block slows later kernels on older buffers by a third
        ybar = Td - Td.mean()
        Tbar, Cib = torch.empty_like(Td), torch.zeros_like(Td)
        def adj10():
            for _ in range(10):
                api.adjoint(Tbar, Cib, ybar, Td, Cf, 1.0, dt, inv, ci_scaled=scaled)
        t_adj = timed(adj10, reps=3) / 10
        out[f"adjoint_256_{name}_ms"] = round(1e3 * t_adj, 4)
        out[f"adjoint_256_{name}_gbs"] = round(6 * n ** 3 * Td.element_size() / t_adj / 1e9, 1)
        for tag, every in (("sqrt_nt", ag.default_every(nt)), ("all_states", 1)):
            t_grad = timed(lambda: ag.loss_and_grad(Td, Cd, Tobs, 1.0, dt, inv, nt, every=every), reps=2)
            out[f"grad_256_{name}_{tag}_ms"] = round(1e3 * t_grad, 2)
            out[f"grad_over_fwd_256_{name}_{tag}"] = round(t_grad / t_fwd, 3)
            if t_fwd2 is not None:
                out[f"grad_over_fwd2_256_{name}_{tag}"] = round(t_grad / t_fwd2, 3)
            torch.cuda.empty_cache()
        del Td, Ctd, Cd, Cf, a, b, Tobs, fa, fb, ybar, Tbar, Cib
        api.clear_graph_cache()
        torch.cuda.empty_cache()

    # 2-D form of the step (z term dropped): FP64 16384^2 on the pre-scaled coefficient and
    # FP32 32768^2 in deviation storage, nt = 100, graph-captured; T_eff = 3 n^2 elem nt / t
    for name, n2, dtype in (("fp64", 16384, torch.float64), ("fp32", 32768, torch.float32)):
        T2d, C2d, dt2, inv2, scaled2 = fields2d(torch, api, inputs, n2, dtype, dev)
        U2d = torch.empty_like(T2d)
        t = timed(lambda: api.run2d(T2d, U2d, C2d, 1.0, dt2, inv2, 100, graph=True, ci_scaled=scaled2))
        out[f"diffusion2d_{name}_{n2}_teff_gbs"] = round(3 * n2 * n2 * T2d.element_size() * 100 / t / 1e9, 1)
        del T2d, C2d, U2d
        api.clear_graph_cache()
        torch.cuda.empty_cache()

    # batched workload: 256 problems, n_p uniform in {32..160}, nt = 500, one launch
    # per step (graph-captured): the TMA z-march on padded rows (tuned z-chunks; FP64 on
    # Ci as given and on the pre-scaled coefficient), the column march on contiguous
    # fields, and one launch per problem
    from paper_2211_15634_gb300 import tuner
    sizes = inputs.batch_sizes(256)
    nt = 500
    for name, dtype in (("fp64", torch.float64), ("fp32", torch.float32)):
        variants = [("", False)] + ([("_ci_scaled", True)] if dtype == torch.float64 else [])
        for tag, scaled in variants:
            probs, bytes_per_step = batch_workload(torch, api, inputs, dtype, dev, len(sizes),
                                                   pitched=True, ci_scaled=scaled)
            best = tuner.tune(probs, kernel="zmarch", ci_scaled=scaled)  # per size class, cached
            b = tuner.tuned_batch(probs, kernel="zmarch", ci_scaled=scaled)
            t_b = timed(lambda: b.run(nt, graph=True), reps=2)
            out[f"batch_{name}{tag}_teff_gbs"] = round(bytes_per_step * nt / t_b / 1e9, 1)
            out[f"batch_{name}{tag}_tiles"] = {f"{lo}-{hi}": list(t)[2] for (lo, hi), t in sorted(best.items())}
            out[f"batch_{name}{tag}_depth"] = 2 if b.temporal2 else 1  # tuned temporal-block depth
            del probs, b
            api.clear_graph_cache()
            torch.cuda.empty_cache()

        probs, bytes_per_step = batch_workload(torch, api, inputs, dtype, dev, len(sizes))
        b0 = api.Batch(probs, kernel="column")  # library default tile for every problem
        t_0 = timed(lambda: b0.run(nt, graph=True), reps=1)
        out[f"batch_{name}_column_teff_gbs"] = round(bytes_per_step * nt / t_0 / 1e9, 1)
        del b0
        api.clear_graph_cache()

        # one launch per problem, problem-major: each problem's nt steps in a row
        # (its fields stay in the 129 MB L2 across its own steps)
        def per_problem():
            for p in probs:
                api.run(p["T"], p["T2"], p["Ci"], 1.0, p["dt"], p["inv_spacing"], nt)
        t_p = timed(per_problem, reps=1)
        out[f"batch_{name}_per_problem_teff_gbs"] = round(bytes_per_step * nt / t_p / 1e9, 1)

        # one launch per problem, step-major (what one batched launch per step
        # replaces): 50 steps of all problems
        def per_problem_stepwise(nsteps=50):
            for it in range(nsteps):
                for p in probs:
                    src, dst = (p["T"], p["T2"]) if it % 2 == 0 else (p["T2"], p["T"])
                    api.step(dst, src, p["Ci"], 1.0, p["dt"], p["inv_spacing"])
        t_s = timed(per_problem_stepwise, reps=1)
        out[f"batch_{name}_per_problem_stepwise_teff_gbs"] = round(bytes_per_step * 50 / t_s / 1e9, 1)
        del probs
        api.clear_graph_cache()
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2211_15634_gb300 import api, inputs
    from paper_2211_15634_gb300 import autograd as ag
    from paper_2211_15634_gb300 import _lib

    _lib.load()
    n, nt, K, W = args.size, args.nt, args.steps, args.warmup
    assert W >= 3, "need at least 3 warm-up steps"
    T0, Ci, inv = fields(n)
    dev = torch.device(f"cuda:{local}")
    T = torch.from_numpy(T0).to(dev)
    T2 = torch.empty_like(T)
    C = torch.from_numpy(Ci).to(dev)
    Cs = torch.empty_like(C)  # dt*lam*_dx^2*Ci, rebuilt every step from this step's dt
    lam = 1.0
    bytes_per_launch = 3 * n ** 3 * 8
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def one_step(run_events=None):
        dt = api.stable_dt(C, lam)          # A1: maximum(Ci) on the GPU, dt on the host
        api.scale_ci(C, lam, dt, inv, out=Cs)  # one pass: Cs = dt*lam*_dx^2*Ci
        if run_events is not None:
            run_events[0].record()
        # A4: Fig. 1's T2 = copy(T) on the boundary, then the nt steps, replayed from the
        # library's cached CUDA graph (captured in the warm-up)
        api.run(T, T2, Cs, lam, dt, inv, nt, graph=True, ci_scaled=True)
        if run_events is not None:
            run_events[1].record()
        return dt

    def one_step_eager():
        """The same step with nt individual launches (no graph), for comparison."""
        dt = api.stable_dt(C, lam)
        api.scale_ci(C, lam, dt, inv, out=Cs)
        api.copy_boundary(T2, T)
        for it in range(nt):
            src, dst = (T, T2) if it % 2 == 0 else (T2, T)
            api.step(dst, src, Cs, lam, dt, inv, ci_scaled=True)

    for _ in range(W):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local).start() if rank == 0 else None
    rev = [[ev(), ev()] for _ in range(K)]  # around each graph replay (boundary copy + nt steps)
    sev = [[ev(), ev()] for _ in range(K)]  # per-step samples
    torch.cuda.synchronize()
    t_start, t_end = ev(), ev()
    t_start.record()
    for s in range(K):
        sev[s][0].record()
        dt = one_step(rev[s])
        sev[s][1].record()
    t_end.record()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    region_s = t_start.elapsed_time(t_end) / 1e3
    # mean step-kernel duration: each replay's span over its nt launches (the boundary copy
    # kernel in the span is counted against the steps, so this errs low)
    launch_ms = [a.elapsed_time(b) / nt for (a, b) in rev]
    step_ms = [a.elapsed_time(b) for (a, b) in sev]
    region_s = max_over_ranks(region_s, dev)
    gbs = whole_job_rate(bytes_per_launch * nt * K, region_s, world) / 1e9
    # per step: max reduction (2 kernels), coefficient scaling, boundary copy, nt steps
    gpu_launches = K * (nt + 4)

    # the same steps launched one by one (no graph)
    one_step_eager()
    torch.cuda.synchronize()
    g0, g1 = ev(), ev()
    g0.record()
    for _ in range(K):
        one_step_eager()
    g1.record()
    torch.cuda.synchronize()
    eager_gbs = bytes_per_launch * nt * K / (g0.elapsed_time(g1) / 1e3) / 1e9
    api.clear_graph_cache()

    # end to end through the public API: pinned host in, host result out, every step.
    # api.SolvePipeline overlaps step i's computation with step i+1's copies in and
    # step i-1's copy out (two device buffer sets, separate copy streams); the timed
    # region runs from the first copy in to the last copy out.  api.solve (one problem
    # at a time, copies not overlapped) is timed beside it.
    e2e = None
    if rank == 0 or world > 1:
        T0h = torch.from_numpy(T0).pin_memory()
        Cih = torch.from_numpy(Ci).pin_memory()
        outh = torch.empty_like(T0h).pin_memory()
        bufs = (T, T2, C)
        api.solve(T0h, Cih, lam, None, inv, nt, out_host=outh, buffers=bufs)
        t0 = time.perf_counter()
        e2e_steps = max(1, args.e2e_steps if args.e2e_steps > 0 else K)
        for _ in range(e2e_steps):
            api.solve(T0h, Cih, lam, None, inv, nt, out_host=outh, buffers=bufs)
        serial_s = (time.perf_counter() - t0) / e2e_steps
        pipe = api.SolvePipeline(tuple(T0.shape), torch.float64, lam, inv, nt)
        for _ in range(2):  # warm-up: one problem through each of the two buffer sets
            pipe.submit(T0h, Cih, outh)
        pipe.finish()
        steps = e2e_steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            pipe.submit(T0h, Cih, outh)
        pipe.finish()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": round(world * bytes_per_launch * nt * steps / e2e_s / 1e9, 1),
               "unit": "GB/s", "h2d_bytes_per_step": 2 * n ** 3 * 8,
               "d2h_bytes_per_step": n ** 3 * 8, "steps": steps,
               "api": "SolvePipeline (copies overlapped with the neighbouring steps)",
               "solve_one_at_a_time": round(world * bytes_per_launch * nt / serial_s / 1e9, 1)}
        del pipe
        api.clear_graph_cache()

    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0

    hbm, src = measured_peaks()
    mean_launch_s = statistics.mean(launch_ms) / 1e3
    achieved = bytes_per_launch / mean_launch_s / 1e9
    kernel = api.step_kernel_name(T2, T, Cs, lam, dt, inv, ci_scaled=True)
    digest = source_digest(api.step_kernel_sources(kernel))
    traffic = profiled_traffic(kernel, digest, n)
    line = {
        "metric": METRIC, "value": round(gbs, 1), "unit": "GB/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(1e3 * region_s / K, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": round(gbs / world / PAPER_TEFF_A100, 3),
        "vs_baseline_note": "paper T_eff 1262 GB/s, FP64 512^3, A100 SXM4: another machine, context",
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"diffusion3d FP64 {n}^3 Gaussian T0, random Ci, nt={nt}",
                   "nx": n, "ny": n, "nz": n, "nt": nt, "lam": lam, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (3 x 1 GiB fields), no flush needed",
                   "pct_hbm_peak": round(100 * gbs / world / hbm, 1)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": traffic, "kernel": kernel,
                     "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
                     "launches_timed": K * nt,
                     "mean_launch_ms": round(1e3 * mean_launch_s, 4),
                     "timing": "CUDA events around each graph replay, span / nt"},
        "samples": step_samples(step_ms, bytes_per_launch * nt),
        "eager_value": round(eager_gbs, 1),
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(T0, Ci, inv)
        except Exception as exc:  # reported, not fatal
            line["cpu_baseline"] = {"error": str(exc)}
    del T, T2, C, Cs
    torch.cuda.empty_cache()
    if not args.no_secondary and world == 1:
        try:
            line["secondary"] = secondary_metrics(torch, api, ag, inputs, log)
        except Exception as exc:
            line["secondary"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_zslab(args):
    """Weak scaling of one decomposed problem: rank r owns 510 planes of a 512 x 512 x
    (510 N + 2) grid (its local fields are 512^3 with the two halo planes), steps them
    with the pre-scaled FP64 kernel, boundary planes first, and exchanges one plane with
    each neighbour per step over NCCL while its interior steps.  T_eff counts the
    global grid: 3 * nodes * 8 bytes * nt per step."""
    import torch
    import torch.distributed as dist

    from paper_2211_15634_gb300 import api, inputs, zslab
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    n, nt, K, W = args.size, args.nt, args.steps, args.warmup
    nzg = (n - 2) * world + 2
    slab = zslab.ZSlab((nzg, n, n), rank, world)
    dev = torch.device(f"cuda:{local}")
    x = torch.from_numpy(inputs.node_coords(n)).to(dev)
    z = torch.arange(slab.z0 - 1, slab.z1 + 1, device=dev, dtype=torch.float64) / (nzg - 1)
    d2 = (x - 0.5) ** 2
    T0 = 1.7 + torch.exp(-((d2[None, None, :] + d2[None, :, None]) + ((z - 0.5) ** 2)[:, None, None]) / 0.01)
    idx = torch.arange((slab.z0 - 1) * n * n, (slab.z1 + 1) * n * n, device="cpu", dtype=torch.int64)
    C = torch.from_numpy((1.0 / inputs.C0) * (1.0 + 0.5 * inputs.uniform(inputs.SEED_CI, idx.numpy().astype(np.uint64)))
                         .reshape(slab.local_shape)).to(dev)
    dx = 1.0 / (n - 1)
    dt = dx * dx / 1.0 / (1.5 / inputs.C0) / 6.1  # the bound max Ci <= 1.5/c0: one dt for all ranks
    inv = (1.0 / dx,) * 3
    Cs = api.scale_ci(C, 1.0, dt, inv)
    T, T2 = T0.clone(), torch.empty_like(T0)
    ex = zslab.HaloExchange(slab, T, transport="device") if world > 1 else None

    def one():
        T.copy_(T0)
        zslab.run_slab(slab, ex, T, T2, Cs, 1.0, dt, inv, nt, ci_scaled=True)
    for _ in range(W):
        one()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(K):
        one()
    b.record()
    torch.cuda.synchronize()
    t = max_over_ranks(a.elapsed_time(b) / 1e3, dev)
    if rank == 0:
        gbs = 3 * n * n * nzg * 8 * nt * K / t / 1e9
        print(json.dumps({
            "metric": METRIC, "value": round(gbs, 1), "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": round(1e3 * t / K, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"diffusion3d FP64 {n}x{n}x{nzg} z-slabs (one 512^3 slab per rank, "
                                   f"incl. halos), Gaussian T0, random Ci, nt={nt}",
                       "nx": n, "ny": n, "nz": nzg, "nt": nt, "parallelism": f"zslab x{world}",
                       "note": "each timed step includes a reset of T from T0 (one field copy)"}}),
            flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.kernel_loop:
        return run_kernel_loop(args)
    if args.zslab:
        return run_zslab(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
