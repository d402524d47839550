"""Autotuner: picks the fused 2D kernel family (warp march or band march), its tile
height and the fusion depth (steps per launch, temporal blocking) for a handle by
timing candidates on the caller's own buffers, and remembers the choice in a JSON
cache keyed by device, field shapes, element type, passes and options (and whether
the step runs on the compensated FP32 state, whose kernel is the warp march: only its
lane width and tile height are searched).

The cache lives in $MPDATA_GB300_TUNE_CACHE, else
$XDG_CACHE_HOME/mpdata_gb300/autotune.json (~/.cache/... by default).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import capi

# (MPDATA_TUNE_KERNEL, MPDATA_TUNE_TILE_ROWS, MPDATA_TUNE_STEPS_PER_LAUNCH): warp-march tile
# heights (lanes of 4 and of 2 columns), band heights, one step per launch; then fusion depths
# 2..4 (the temporal-blocking kernel, whose tiles are fixed: family and rows do not apply)
CANDIDATES = tuple([(1, r, 1) for r in (0, 6, 8, 12, 16, 24, 32, 48, 64)] +
                   [(3, r, 1) for r in (6, 8, 12, 16, 24, 32)] +
                   [(2, r, 1) for r in (0, 16, 32, 64, 128, 256)] +
                   [(0, 0, d) for d in (2, 3, 4)])
# batched handles (several fields, one persistent launch per step): lanes of 4 or 2 columns and the
# tile height of the work items
BATCH_CANDIDATES = tuple((k, r, 1) for k in (1, 3) for r in (24, 32, 48, 64, 96, 128))
# options the temporal-blocking kernel does not cover
_TBLOCK_EXCLUDED = ("TOT", "ABS", "DFL", "NUG", "KAHAN", "RHS_EULER_A", "RHS_EULER_B", "RHS_TRAPEZ", "STAGED",
                    "OPEN0", "OPEN1", "OPEN2", "SW")
_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("MPDATA_GB300_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "mpdata_gb300", "autotune.json")


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key_of(solver) -> str:
    name = torch.cuda.get_device_name(solver.device)
    shapes = ";".join("x".join(map(str, s)) for s in solver.shapes[:8])
    if len(solver.shapes) > 8:
        shapes += f";+{len(solver.shapes) - 8}fields:{solver.total}"
    return f"{name}|{shapes}|{solver.dtype}|n_iters={solver.n_iters}|opts={solver.opts}"


def tblock_applies(solver) -> bool:
    """Whether the handle's steps can run at a fusion depth above 1: one 2D field, two passes
    and none of the options the temporal-blocking kernel leaves out."""
    excluded = 0
    for name in _TBLOCK_EXCLUDED:
        excluded |= getattr(capi, name)
    return len(solver.shapes) == 1 and len(solver.shapes[0]) == 2 and solver.n_iters == 2 and not (solver.opts & excluded)


def time_steps(solver, psi, gc, g=None, r=None, dt=0.0, steps=20, flush_bytes=256 << 20, depth=1):
    """Seconds per step on the device: each call of `depth` steps (one launch at the handle's
    fusion depth) is bracketed by CUDA events after an L2 flush, all calls are queued before
    one synchronisation (so host launch overhead does not fall inside the events), and the
    per-call times are averaged and divided by `depth`."""
    dev = solver.device
    stream = torch.cuda.current_stream(dev)
    a, b = psi.clone(), torch.empty_like(psi)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev) if flush_bytes else None
    solver.advance(a, b, gc, g, r, dt, 2 * depth)
    fwd = capi.prepare_advance(solver.h, a, b, gc, g, r, dt, depth)
    bwd = capi.prepare_advance(solver.h, b, a, gc, g, r, dt, depth)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k, (e0, e1) in enumerate(evs):
        if flush is not None:
            flush.zero_()
        e0.record(stream)
        (fwd if k % 2 == 0 else bwd)()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3 / steps / depth


def time_steps_comp(solver, hi, lo, gc, g=None, r=None, dt=0.0, steps=20, flush_bytes=256 << 20):
    """time_steps for mpdata_advance_compensated on the state hi + lo."""
    dev = solver.device
    stream = torch.cuda.current_stream(dev)
    a, al = hi.clone(), lo.clone()
    b, bl = torch.empty_like(hi), torch.empty_like(lo)
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev) if flush_bytes else None
    solver.advance_compensated(a, al, b, bl, gc, g, r, dt, 2)
    fwd = capi.prepare_advance_compensated(solver.h, a, al, b, bl, gc, g, r, dt, 1)
    bwd = capi.prepare_advance_compensated(solver.h, b, bl, a, al, gc, g, r, dt, 1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k, (e0, e1) in enumerate(evs):
        if flush is not None:
            flush.zero_()
        e0.record(stream)
        (fwd if k % 2 == 0 else bwd)()
        e1.record(stream)
    torch.cuda.synchronize(dev)
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3 / steps


def _apply(solver, choice):
    kernel, rows, depth = choice
    solver.tune(capi.TUNE_KERNEL, int(kernel))
    solver.tune(capi.TUNE_TILE_ROWS, int(rows))
    solver.tune(capi.TUNE_STEPS_PER_LAUNCH, int(depth))


def autotune(solver, psi, gc, g=None, r=None, dt=0.0, candidates=CANDIDATES, steps=20, use_cache=True,
             flush_bytes=256 << 20, lo=None):
    """Choose (MPDATA_TUNE_KERNEL, MPDATA_TUNE_TILE_ROWS, MPDATA_TUNE_STEPS_PER_LAUNCH) for
    `solver` (an Mpdata handle); returns ((kernel, tile_rows, depth), seconds per step,
    {candidate: seconds}).  The handle is left tuned to the winner.  Fusion depths above 1 are
    tried only where the temporal-blocking kernel covers the handle, and are timed per step
    over calls of `depth` steps.  Batched handles search BATCH_CANDIDATES by default.  With lo (the low parts of a compensated FP32 state psi = hi +
    lo) the compensated step is timed, over the warp-march candidates at depth 1."""
    key = key_of(solver) + ("|compensated" if lo is not None else "")
    if len(solver.shapes) > 1 and candidates is CANDIDATES:
        candidates = BATCH_CANDIDATES
    if lo is not None:
        candidates = tuple(c for c in candidates if c[0] in (1, 3) and c[2] == 1)
    if solver.dtype != torch.float32:
        candidates = tuple(c for c in candidates if c[0] != 3)
    if not tblock_applies(solver):
        candidates = tuple(c for c in candidates if c[2] == 1)
    if use_cache:
        with _lock:
            hit = _load_cache().get(key)
        if hit is not None:
            choice = (int(hit.get("kernel", 0)), int(hit["tile_rows"]), int(hit.get("steps_per_launch", 1)))
            _apply(solver, choice)
            return choice, float(hit["seconds_per_step"]), {}
    timings = {}
    for c in candidates:
        _apply(solver, c)
        if lo is not None:
            timings[c] = time_steps_comp(solver, psi, lo, gc, g, r, dt, steps, flush_bytes)
        else:
            timings[c] = time_steps(solver, psi, gc, g, r, dt, steps, flush_bytes, depth=c[2])
    best = min(timings, key=timings.get)
    _apply(solver, best)
    if use_cache:
        with _lock:
            cache = _load_cache()
            cache[key] = {"kernel": int(best[0]), "tile_rows": int(best[1]), "steps_per_launch": int(best[2]),
                          "seconds_per_step": timings[best]}
            _store_cache(cache)
    return best, timings[best], timings
