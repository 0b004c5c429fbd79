"""Autotuner for the batched launch: kernel and tile shape.

For a set of lattice shapes and a storage type it times the batched step of a
scratch batch of the same shapes (CUDA events on the batch's stream, after
warm-up steps) for every candidate configuration and picks the fastest.  A
configuration is the kernel -- cells per thread (1, or 2 on packed FP32) and
time steps per launch (1, or 2 through shared memory on two-step tiles) --
and, for one-step launches, the tile shape.  Results are cached per (GPU name,
storage, shape signature) in a JSON file, by default
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
# (cells per thread, steps per launch) of the batched kernels; FP64 has only the first
KERNELS = [(1, 1), (2, 1), (2, 2)]
TWO_STEP_TILE = (64, 16)  # the tile of the two-step kernel (fixed by its shared-memory layout)


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


def configurations(storage: str, candidates=CANDIDATES, kernels=KERNELS):
    """Every (cells, steps_per_launch, tile_x, tile_y) to try for a storage."""
    out = []
    for cells, spl in kernels:
        if storage == "f64" and (cells, spl) != (1, 1):
            continue
        if spl == 2:
            out.append((cells, spl) + TWO_STEP_TILE)
        else:
            out.extend((cells, spl, tx, ty) for tx, ty in candidates)
    return out


def measure(shapes, storage="f32", configs=None, steps=64, warmup=32):
    """Seconds per batched step for each configuration (see configurations)."""
    import torch

    from .batch import Batch

    configs = configurations(storage) if configs is None else configs
    stream = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(stream):
        b = Batch(storage, stream=stream)
        for nx, ny in shapes:
            i = b.add(nx, ny, steps=1 << 40, s=1.99, variant="II",
                      chi_x=[0.1] * min(8, nx) + [0.0] * (nx - min(8, nx)),
                      chi_y=[0.0] * ny)
            b.init_equilibrium(i, np.ones((ny, nx)), 0.0, 0.0)
        for cells, spl, tx, ty in configs:
            b.configure(cells, spl, (tx, ty))
            b.step(warmup)
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.step(steps)
            z.record(stream)
            z.synchronize()
            out[(cells, spl, tx, ty)] = a.elapsed_time(z) / 1e3 / steps
        b.close()
    return out


def tuned_config(shapes, storage="f32", retune=False, configs=None) -> dict:
    """Fastest {"cells", "steps_per_launch", "tile"} for this shape set, from the
    cache or measured."""
    import torch

    key = f"{torch.cuda.get_device_name()}|{storage}|kernel+tile|{signature(shapes)}"
    cache = _load()
    if not retune and key in cache:
        c = cache[key]
        return {"cells": c["cells"], "steps_per_launch": c["steps_per_launch"],
                "tile": tuple(c["tile"])}
    times = measure(shapes, storage, configs)
    cells, spl, tx, ty = min(times, key=times.get)
    cache[key] = {"cells": cells, "steps_per_launch": spl, "tile": [tx, ty],
                  "seconds_per_step": {f"cells{c}/spl{s}/{a}x{b}": t
                                       for (c, s, a, b), t in times.items()}}
    _store(cache)
    return {"cells": cells, "steps_per_launch": spl, "tile": (tx, ty)}


def tuned_tiling(shapes, storage="f32", retune=False):
    """Tile shape of the tuned configuration (for callers that only set the
    tiling)."""
    return tuned_config(shapes, storage, retune)["tile"]
