"""Tile-shape autotuner for the batched step.

Problems are grouped into size classes by their largest extent; for each class
the batched kernel is timed (CUDA events, a few steps after warm-up) on the
whole batch with every candidate work-item shape (tile_x, tile_y, tile_z) for
that class, and the fastest shape is kept.  The candidates depend on the kernel
the batch runs: the column march takes x-y tiles and z-chunks, the TMA z-march
(fixed x-y tiles) its z-chunk length.  For a z-march batch that can run fused
step pairs (FP32, or FP64 on the pre-scaled coefficient) the temporal-block
depth (1 or 2 steps per pass) is then chosen for the whole batch by timing both
with the tuned z-chunks.  Results are cached as JSON keyed by GPU name, dtype,
kernel and size class (and "depth"; file ``$PS_TUNER_CACHE`` or
``~/.cache/psdiff/tuner.json``), so later runs reuse them without timing.
``tuned_batch`` builds the final table with each problem's class shape and the
chosen depth.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import api

Tile = Tuple[int, int, int]

# Candidate work-item shapes (tile_x, tile_y, tile_z): tile_x * tile_y columns,
# each marched over tile_z planes.  tile_x == 0 is a row-packed rule: the item
# spans whole interior rows (no partly idle warps at row ends) and as many rows
# as make about tile_y columns.
DEFAULT: Tile = (32, 8, 32)  # the library's default work item (batch_default_tile)
CANDIDATES: List[Tile] = [DEFAULT, (32, 8, 16), (32, 8, 64), (32, 16, 16), (64, 4, 32),
                          (0, 256, 16), (0, 256, 32), (0, 512, 16), (0, 512, 32)]


def tile_for(problem, cand: Tile) -> Tile:
    """Concrete (tile_x, tile_y, tile_z) of a candidate for one problem."""
    tx, ty, tz = cand
    if tx != 0 or ty == 0:  # a fixed shape, or a z-march candidate (x-y tile ignored)
        return cand
    row = problem["T"].shape[2] - 2
    rows = max(1, min(problem["T"].shape[1] - 2, -(-ty // row)))
    while row * rows > 4096:
        rows -= 1
    return row, rows, tz
# z-march candidates: planes per work item (the x-y tile is the kernel's own)
ZMARCH_DEFAULT: Tile = (0, 0, 64)
ZMARCH_CANDIDATES: List[Tile] = [ZMARCH_DEFAULT, (0, 0, 16), (0, 0, 32), (0, 0, 128)]

SIZE_CLASSES: List[Tuple[int, int]] = [(3, 48), (48, 80), (80, 112), (112, 144), (144, 1 << 30)]


def cache_path() -> str:
    return os.environ.get("PS_TUNER_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "psdiff", "tuner.json"))


def _load_cache() -> Dict[str, list]:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save_cache(c: Dict[str, list]) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only costs re-tuning


def size_class(p) -> Tuple[int, int]:
    n = max(p["T"].shape)
    for lo, hi in SIZE_CLASSES:
        if lo <= n < hi:
            return lo, hi
    return SIZE_CLASSES[-1]


def _key(device, dtype, cls, kernel="column", ci_scaled=False) -> str:
    name = torch.cuda.get_device_name(device)
    kern = kernel + ("-scaled" if ci_scaled else "")
    return f"{name}|{'f64' if dtype == torch.float64 else 'f32'}|{kern}|{cls[0]}-{cls[1]}"


def batch_kernel(problems, kernel: str = "auto", ci_scaled: bool = False) -> str:
    """The kernel ("column" or "zmarch") a Batch of these problems would run."""
    return api.Batch(problems, kernel=kernel, ci_scaled=ci_scaled, prescale=False).kernel


def prescaled(problems, kernel: str = "auto", ci_scaled: bool = False):
    """(problems, ci_scaled) as an api.Batch would step them: FP64 problems on Ci as
    given get their pre-scaled copy once here (see api.Batch's ``prescale``), so that
    the candidates timed below do not each make their own."""
    if not ci_scaled and api.Batch._prescalable(problems, kernel):
        return [dict(p, Ci=api.Batch._scaled_copy(p)) for p in problems], True
    return problems, ci_scaled


def time_batch_step(problems, cand: Tile, reps: int = 5, warmup: int = 2, kernel: str = "auto",
                    ci_scaled: bool = False) -> float:
    """Milliseconds per batched step of these problems with one candidate shape."""
    b = api.Batch([dict(p, tile=tile_for(p, cand)) for p in problems], kernel=kernel,
                  ci_scaled=ci_scaled)
    for _ in range(warmup):
        b.step(0)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for i in range(reps):
        b.step(i & 1)
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps


def _time_assignment(problems, assign: Dict[Tuple[int, int], Tile], reps: int, kernel: str,
                     ci_scaled: bool) -> float:
    tagged = [dict(p, tile=tile_for(p, assign[size_class(p)])) for p in problems]
    b = api.Batch(tagged, kernel=kernel, ci_scaled=ci_scaled)
    for _ in range(2):
        b.step(0)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for i in range(reps):
        b.step(i & 1)
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / reps


def tune(problems, candidates: Optional[Sequence[Tile]] = None, reps: int = 5,
         use_cache: bool = True, sweeps: int = 2, kernel: str = "auto",
         ci_scaled: bool = False) -> Dict[Tuple[int, int], Tile]:
    """Best tile per size class present in ``problems`` (cached).

    Coordinate descent on the whole batch: classes interact (they share the
    GPU's CTAs and the memory system), so each class's candidates are timed
    with every other class held at its current choice, starting from the
    library default, for ``sweeps`` passes over the classes.  ``candidates``
    defaults to the list of the kernel the batch runs (``kernel``, as for
    :class:`api.Batch`).
    """
    if not problems:
        return {}
    problems, ci_scaled = prescaled(problems, kernel, ci_scaled)
    dev = problems[0]["T"].device
    dtype = problems[0]["T"].dtype
    kern = batch_kernel(problems, kernel, ci_scaled)
    zm = kern == "zmarch"
    if candidates is None:
        candidates = ZMARCH_CANDIDATES if zm else CANDIDATES
    start = ZMARCH_DEFAULT if zm else DEFAULT
    cache = _load_cache() if use_cache else {}
    classes = sorted({size_class(p) for p in problems})
    keys = {cls: _key(dev, dtype, cls, kern, ci_scaled) for cls in classes}
    if all(keys[c] in cache for c in classes):
        return {c: tuple(cache[keys[c]]) for c in classes}
    assign = {c: start for c in classes}
    best_t = _time_assignment(problems, assign, reps, kernel, ci_scaled)
    for _ in range(sweeps):
        improved = False
        for c in classes:
            for cand in candidates:
                if cand == assign[c]:
                    continue
                trial = dict(assign)
                trial[c] = cand
                t = _time_assignment(problems, trial, reps, kernel, ci_scaled)
                if t < best_t * 0.99:  # keep only clear wins
                    assign, best_t, improved = trial, t, True
        if not improved:
            break
    for c in classes:
        cache[keys[c]] = list(assign[c])
    if use_cache:
        _save_cache(cache)
    return assign


def _time_pairs(problems, assign, reps: int, kernel: str, ci_scaled: bool) -> float:
    """Milliseconds per step with fused pairs (one launch per two steps)."""
    tagged = [dict(p, tile=tile_for(p, assign[size_class(p)])) for p in problems]
    b = api.Batch(tagged, kernel=kernel, ci_scaled=ci_scaled, temporal2=True)
    for _ in range(2):
        b.step2(0)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for i in range(reps):
        b.step2(i & 1)
    e.record()
    e.synchronize()
    return s.elapsed_time(e) / (2 * reps)


def pairs_possible(problems, kernel: str = "auto", ci_scaled: bool = False) -> bool:
    """Whether these problems can run fused step pairs on the z-march."""
    if batch_kernel(problems, kernel, ci_scaled) != "zmarch":
        return False
    return problems[0]["T"].dtype == torch.float32 or ci_scaled


def tune_depth(problems, reps: int = 5, use_cache: bool = True, kernel: str = "auto",
               ci_scaled: bool = False, **kw) -> int:
    """Temporal-block depth (1 or 2 steps per pass) for the whole batch, timed with
    each class's tuned z-chunk (cached)."""
    if not problems:
        return 1
    problems, ci_scaled = prescaled(problems, kernel, ci_scaled)
    if not pairs_possible(problems, kernel, ci_scaled):
        return 1
    dev = problems[0]["T"].device
    dtype = problems[0]["T"].dtype
    key = _key(dev, dtype, ("depth", "all"), "zmarch", ci_scaled)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return int(cache[key][0])
    assign = tune(problems, reps=reps, use_cache=use_cache, kernel=kernel, ci_scaled=ci_scaled, **kw)
    t1 = _time_assignment(problems, assign, reps, kernel, ci_scaled)
    t2 = _time_pairs(problems, assign, reps, kernel, ci_scaled)
    depth = 2 if t2 < 0.99 * t1 else 1  # keep only a clear win
    if use_cache:
        cache = _load_cache()
        cache[key] = [depth]
        _save_cache(cache)
    return depth


def tuned_batch(problems, kernel: str = "auto", ci_scaled: bool = False, depth=None, **kw) -> api.Batch:
    """A Batch whose problems carry the tuned tile of their size class, stepping at the
    tuned temporal-block depth (``depth`` = 1 or 2 overrides it).  Tuning times real
    steps on the problems' own fields (unless every choice is cached): set their
    states after this call."""
    problems, ci_scaled = prescaled(problems, kernel, ci_scaled)
    best = tune(problems, kernel=kernel, ci_scaled=ci_scaled, **kw)
    if depth is None:
        depth = tune_depth(problems, kernel=kernel, ci_scaled=ci_scaled, **kw)
    tagged = [dict(p, tile=tile_for(p, best[size_class(p)])) for p in problems]
    return api.Batch(tagged, kernel=kernel, ci_scaled=ci_scaled, temporal2=depth == 2)
