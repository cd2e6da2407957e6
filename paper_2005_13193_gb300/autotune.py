"""Brick-shape and brick-kernel autotuner.

The brick is the unit of reuse of the binned kernels: one thread block stages
a brick's coefficients plus the 3-node stencil halo in shared memory and
interpolates every particle binned into it.  Larger bricks re-read less halo
per particle but hold fewer blocks per SM; the best shape depends on the grid,
the particle density and the coefficient type, so it is measured, on the
caller's own data, by timing the real step for each candidate.

`tune_tracker` picks (brick kernel, brick shape) for single-field Heun steps
and applies the kernel choice with ps_tune_set; `tune_batch` picks the brick
shape of a many-field plan.  Both can write the choice to a small text cache,
one "key values" pair per line, which ps_batch_plan reads back ("brick bx by
bz"); `load_cache` reads it in Python.
"""
from __future__ import annotations

import os
from typing import Iterable, Optional

import torch

from . import BatchPlan, PSError, SplineField, Tracker, ps_tune_get, ps_tune_set

# brick shapes (x, y, z) tried by default: powers of two the grids of the
# workloads divide, from 64 to 2048 cells, x extents that keep the halo row
# within 32 nodes
CANDIDATES = ((8, 8, 8), (8, 8, 4), (8, 4, 4), (4, 4, 4), (8, 8, 16), (16, 8, 8),
              (16, 8, 4), (16, 16, 8))
KERNELS = (0, 2, 5)


def _time_ms(fn, warmup: int, reps: int, stream=None) -> float:
    for _ in range(warmup):
        fn()
    s = stream or torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps


def write_cache(path: str, entries: dict, comment: str = "") -> None:
    """Write {key: tuple of ints} as "key v0 v1 ..." lines (atomic replace)."""
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        if comment:
            for line in comment.splitlines():
                f.write(f"# {line}\n")
        for k, v in entries.items():
            vals = v if isinstance(v, (tuple, list)) else (v,)
            f.write(k + " " + " ".join(str(int(x)) for x in vals) + "\n")
    os.replace(tmp, path)


def load_cache(path: str) -> dict:
    out = {}
    if not path or not os.path.exists(path):
        return out
    with open(path) as f:
        for line in f:
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            try:
                out[parts[0]] = tuple(int(x) for x in parts[1:])
            except ValueError:
                continue
    return out


def tune_tracker(field: SplineField, pos: torch.Tensor, dt: float = 1e-3,
                 candidates: Iterable = CANDIDATES, kernels: Iterable = KERNELS,
                 steps: int = 2, warmup: int = 1, cache: Optional[str] = None,
                 apply: bool = True):
    """Time `steps` re-binned Heun steps of `pos` through `field` for every
    (kernel, brick) pair; `pos` is left unchanged.  Returns (best, table) with
    best = (kernel, brick) and table = {(kernel, brick): ms per step}.  With
    apply=True the best kernel is set process-wide (ps_tune_set)."""
    old_kernel = ps_tune_get("brick_kernel")
    table = {}
    try:
        for k in kernels:
            ps_tune_set("brick_kernel", int(k))
            for b in candidates:
                b = tuple(int(v) for v in b)
                try:
                    tr = Tracker(field, pos.clone(), brick=b, keep_velocity=False)
                    table[(int(k), b)] = _time_ms(lambda: tr.step(dt), warmup, steps)
                except PSError:
                    continue  # shape not supported (e.g. halo above shared memory)
                finally:
                    tr = None
    finally:
        ps_tune_set("brick_kernel", old_kernel)
    if not table:
        raise RuntimeError("no candidate brick ran")
    best = min(table, key=table.get)
    if apply:
        ps_tune_set("brick_kernel", best[0])
    if cache:
        write_cache(cache, {"kernel": best[0], "brick": best[1]},
                    comment=f"tracker: {table[best]:.4f} ms per step, grid {field.n}")
    return best, table


def tune_batch(grids, nps, fields, pos: torch.Tensor, coef_dtype=torch.float32,
               dt: float = 1e-3, candidates: Iterable = CANDIDATES, steps: int = 2,
               warmup: int = 1, cache: Optional[str] = None):
    """Time `steps` eager batched Heun steps for every candidate brick shape;
    `pos` is left unchanged.  `fields` is the list BatchPlan.run takes.
    Returns (best brick, {brick: ms per step})."""
    table = {}
    for b in candidates:
        b = tuple(int(v) for v in b)
        try:
            plan = BatchPlan(grids, nps, coef_dtype=coef_dtype, brick=b)
        except PSError:
            continue
        p = pos.clone()
        try:
            table[b] = _time_ms(
                lambda: plan.run(fields, p, 1, dt, solve=False, use_graph=False),
                warmup, steps)
        except PSError:
            pass
        finally:
            del plan, p
    if not table:
        raise RuntimeError("no candidate brick ran")
    best = min(table, key=table.get)
    if cache:
        write_cache(cache, {"brick": best},
                    comment=f"batch of {len(grids)} fields: {table[best]:.4f} ms per step")
    return best, table
