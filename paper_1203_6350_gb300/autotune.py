"""Tile-shape autotuner for the batched launch.

For a set of lattice shapes and a storage type it times the batched step with
each candidate tile shape on a scratch batch of the same shapes (CUDA events
on the batch's stream, after warm-up steps) and picks the fastest.  Results
are cached per (GPU name, storage, cells per thread, shape signature) in a
JSON file, by default
~/.cache/lbm_gb300/autotune.json (LBM_AUTOTUNE_CACHE overrides it).
"""
from __future__ import annotations

import json
import math
import os
from collections import Counter

import numpy as np

CANDIDATES = [(32, 8), (32, 16), (64, 8), (64, 16), (128, 8), (128, 16), (128, 32), (128, 64),
              (256, 4), (256, 8), (256, 16)]


def cache_path() -> str:
    return os.environ.get("LBM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300",
                                       "autotune.json"))


def signature(shapes) -> str:
    """Order-free summary of a shape set: counts per (log2 nx, log2 ny) bucket."""
    c = Counter((int(math.log2(max(1, nx))), int(math.log2(max(1, ny)))) for nx, ny in shapes)
    return ";".join(f"{a}x{b}:{n}" for (a, b), n in sorted(c.items()))


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, p)


def default_cells(storage: str) -> int:
    """Cells per thread a new batch of this storage uses (see lbm_batch_create)."""
    env = os.environ.get("LBM_CPT")
    if storage == "f64" or env == "1":
        return 1
    if env == "2":
        return 2
    return 2 if storage in ("f16dev", "bf16dev") else 1


def measure(shapes, storage="f32", candidates=CANDIDATES, steps=64, warmup=32, cells=None):
    """Seconds per batched step for each candidate tile shape (cells = cells per
    thread of the batched kernel; None: the batch's default)."""
    import torch

    from .batch import Batch

    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        b = Batch(storage, stream=stream)
        if cells is not None:
            b.cells_per_thread = cells
        for nx, ny in shapes:
            i = b.add(nx, ny, steps=1 << 40, s=1.99, variant="II",
                      chi_x=[0.1] * min(8, nx) + [0.0] * (nx - min(8, nx)),
                      chi_y=[0.0] * ny)
            b.init_equilibrium(i, np.ones((ny, nx)), 0.0, 0.0)
        for tx, ty in candidates:
            b.set_tiling(tx, ty)
            b.step(warmup)
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.step(steps)
            z.record(stream)
            z.synchronize()
            out[(tx, ty)] = a.elapsed_time(z) / 1e3 / steps
        b.close()
    return out


def tuned_tiling(shapes, storage="f32", retune=False, candidates=CANDIDATES, cells=None):
    """Best (tile_x, tile_y) for this shape set and kernel (cells per thread;
    None: the batch's default), from the cache or measured."""
    import torch

    cells = default_cells(storage) if cells is None else cells
    key = f"{torch.cuda.get_device_name()}|{storage}|cpt{cells}|{signature(shapes)}"
    cache = _load()
    if not retune and key in cache:
        return tuple(cache[key]["tile"])
    times = measure(shapes, storage, candidates, cells=cells)
    best = min(times, key=times.get)
    cache[key] = {"tile": list(best), "seconds_per_step": {f"{a}x{b}": t for (a, b), t in
                                                           times.items()}}
    _store(cache)
    return best
