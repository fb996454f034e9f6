"""Tile autotuner for the stencil solvers.

The stencil tile engine has two shape parameters: rows of 32 nodes per tile
(= warps per block, 4 / 8 / 16) and z planes per work item.  Their best values
depend on the grid size, the dimension, the operator, the solver and the GPU.
This module times short fixed-iteration solves (tol = 0, so every candidate
does exactly the same arithmetic work) for each candidate shape with CUDA
events, keeps the fastest, and caches the winner in a JSON file keyed by

    GPU name | solver | operator kind | dimension | size bucket | dtype | team

where the size bucket is the grid's largest side rounded to a power of two and
`team` is "grid" (standalone solve on every co-resident block) or "1" (a
single block, the condition of a small system in the batched solver's queue).

Cache file: $HSOLVE_TUNE_CACHE, else ~/.cache/hsolve/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import _lib
from .solvers import Operator, bicgstab, cg, jacobi

_LOCK = threading.Lock()

ROW_CANDIDATES = (4, 8, 16)
PLANE_CANDIDATES = (0, 8, 16, 32, 64)


def cache_path() -> str:
    return os.environ.get("HSOLVE_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "hsolve",
                                                               "tune.json")


def size_bucket(shape: Sequence[int]) -> int:
    side = max(int(s) for s in shape)
    return 1 << max(0, int(round(math.log2(max(side, 1)))))


def tune_key(gpu: str, solver: str, op_kind: str, shape: Sequence[int], dtype: str, team: str) -> str:
    return "%s|%s|%s|%dd|n%d|%s|team%s" % (gpu, solver, op_kind, len(shape), size_bucket(shape), dtype, team)


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict], path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu_name(device) -> str:
    return torch.cuda.get_device_name(device)


def _operator(shape, op_kind: str, device):
    if op_kind == "laplacian":
        return Operator.laplacian(shape), None
    if op_kind == "upwind":
        from .inputs import upwind_beta
        return Operator.upwind(shape, upwind_beta(shape, 0.5)), None
    if op_kind == "diffusion":
        from .inputs import log_k
        k = torch.from_numpy(np.exp(log_k(shape, 1.0, 0))).to(device)
        return Operator.diffusion(shape, k), k
    raise ValueError(op_kind)


def measure(shape, op_kind: str, solver: str, rows: int, planes: int, team: str = "grid", iters: int = 20,
            reps: int = 3, dtype=torch.float64, device="cuda") -> float:
    """Median milliseconds per iteration of a fixed-iteration solve with the given tile shape."""
    from .inputs import rhs_uniform
    A, _k = _operator(shape, op_kind, device)
    b = torch.from_numpy(rhs_uniform(shape, 0)).to(device=device, dtype=dtype)
    fn = {"cg": cg, "bicgstab": bicgstab, "jacobi": jacobi}[solver]
    kw = dict(tile_rows=rows, tile_planes=planes, max_blocks=1 if team == "1" else 0, true_residual=False,
              timeout_s=30.0)
    if solver in ("cg", "bicgstab"):
        kw.update(tol=0.0, history=False)
    stream = torch.cuda.current_stream(device)
    times = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = fn(A, b, maxit=iters, **kw)
        e1.record(stream)
        torch.cuda.synchronize(device)
        if info.status_code < 0:
            return float("inf")
        if r > 0:
            times.append(e0.elapsed_time(e1) / max(info.iters, 1))
    return float(np.median(times))


def tune(shape, op_kind: str, solver: str, team: str = "grid", dtype=torch.float64, rows=None, planes=None,
         iters: int = 20, device="cuda", path: Optional[str] = None, force: bool = False) -> dict:
    """Times every candidate tile shape and caches the fastest; returns the cache entry."""
    dname = "f64" if dtype == torch.float64 else "f32"
    key = tune_key(_gpu_name(device), solver, op_kind, shape, dname, team)
    with _LOCK:
        cache = load_cache(path)
        if not force and key in cache:
            return cache[key]
    rows = rows or (ROW_CANDIDATES if team == "grid" else (8,))
    nz = shape[2] if len(shape) >= 3 else 1
    planes = planes or tuple(p for p in PLANE_CANDIDATES if p == 0 or p < nz)
    trials = []
    for r in rows:
        for p in planes:
            ms = measure(shape, op_kind, solver, r, p, team, iters, dtype=dtype, device=device)
            trials.append({"tile_rows": r, "tile_planes": p, "ms_per_iter": ms})
    best = min(trials, key=lambda t: t["ms_per_iter"])
    entry = {"tile_rows": best["tile_rows"], "tile_planes": best["tile_planes"],
             "ms_per_iter": best["ms_per_iter"], "trials": trials, "shape": list(shape)}
    with _LOCK:
        cache = load_cache(path)
        cache[key] = entry
        save_cache(cache, path)
    return entry


def lookup(shape, op_kind: str, solver: str, team: str = "grid", dtype=torch.float64, device="cuda",
           path: Optional[str] = None) -> Optional[dict]:
    """The cached entry for this configuration, or None."""
    dname = "f64" if dtype == torch.float64 else "f32"
    key = tune_key(_gpu_name(device), solver, op_kind, shape, dname, team)
    return load_cache(path).get(key)


SMALL_BUCKET = 64


def batch_tile_planes(ops: Sequence[Operator], solvers: Sequence[str], tune_missing: bool = True,
                      device="cuda", path: Optional[str] = None) -> list:
    """Per-system z planes for a batch.  Systems up to SMALL_BUCKET nodes per
    side (the ones the batched solver runs on single blocks from its queue) take
    the team-of-one tuning of their (solver, operator, dimension, size bucket),
    tuned on a representative grid of the bucket when missing; larger systems,
    which run on multi-block teams, keep the cost model (0)."""
    out = []
    done = {}
    for A, s in zip(ops, solvers):
        if s == "mixed":   # tuned as its inner solver
            s = "bicgstab" if A.kind == "upwind" else "cg"
        if size_bucket(A.shape) > SMALL_BUCKET:
            out.append(0)
            continue
        rep = tuple([size_bucket(A.shape)] * len(A.shape))
        key = (s, A.kind, len(A.shape), rep)
        if key not in done:
            entry = lookup(rep, A.kind, s, "1", device=device, path=path)
            if entry is None and tune_missing:
                entry = tune(rep, A.kind, s, "1", device=device, path=path, iters=10)
            done[key] = 0 if entry is None else int(entry["tile_planes"])
        out.append(done[key])
    return out
