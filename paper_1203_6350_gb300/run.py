"""Run one lattice case through the C ABI and report its throughput.

    python -m paper_1203_6350_gb300.run --side 4096 --storage f32 --steps 200

Square lattice at rest (optionally with a centred pulse) with a ramped
absorbing layer; prints one JSON line with MLUPS, algorithmic GB/s
(bytes/cell per launch x cells x launches / time: one launch moves each
population in and out once, whether it advances one time step or two) and
the fraction of the measured HBM copy bandwidth.  Timing uses CUDA events on the lattice's stream after
warm-up steps; the state is larger than L2 for sides >= 2048 in FP32.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_CELL = {"f64": 144, "f32": 72, "f16dev": 36, "bf16dev": 36}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--storage", default="f32", choices=list(BYTES_PER_CELL))
    ap.add_argument("--variant", default="II", choices=["none", "I", "II", "III", "viscous"])
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--width", type=int, default=128)
    ap.add_argument("--pulse", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="run this many copies of the lattice through the batched path")
    ap.add_argument("--tile", default=None, help="batched tile shape, e.g. 128x16")
    ap.add_argument("--cells", type=int, default=None, choices=[1, 2],
                    help="cells per thread (default: the library's choice)")
    ap.add_argument("--per-launch", type=int, default=None, choices=[1, 2],
                    help="time steps per launch (default: the library's choice)")
    ap.add_argument("--arithmetic", default="native", choices=["native", "compensated"],
                    help="collision arithmetic (compensated: FP32 storage, float-float)")
    ap.add_argument("--tma", type=int, default=None, choices=[0, 1],
                    help="TMA staging of two-step launches (default: the library's choice)")
    args = ap.parse_args(argv)

    import torch

    import workloads as wl
    from paper_1203_6350_gb300 import lbm

    w = wl.quiescent(args.side, storage=args.storage, steps=args.steps, width=args.width,
                     variant=args.variant, pulse=args.pulse)
    stream = torch.cuda.Stream()
    copies = max(1, args.batch)
    with torch.cuda.stream(stream):
        if args.batch:
            from paper_1203_6350_gb300.batch import Batch

            tiling = tuple(int(v) for v in args.tile.split("x")) if args.tile else None
            lat = Batch(args.storage, stream=stream, tiling=tiling)
            ids = [lat.add_workload(w, steps=1 << 40, init="pulse") for _ in range(copies)]
        else:
            lat = lbm.Lattice.from_workload(w, stream=stream, init="pulse")
        if args.cells is not None:
            lat.cells_per_thread = args.cells
        if args.per_launch is not None:
            lat.steps_per_launch = args.per_launch
        if args.arithmetic != "native":
            lat.arithmetic = args.arithmetic
        if args.tma is not None and not args.batch:
            lat.tma_staging = bool(args.tma)
        spl = lat.steps_per_launch
        lat.step(args.warmup)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(args.steps)
        b.record(stream)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    cells = w.cells * args.steps * copies
    gbs = BYTES_PER_CELL[args.storage] * cells / spl / t / 1e9
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peak = float(json.load(open(p))["hbm_gbs"])
    d = lat.diagnostics(ids[0]) if args.batch else lat.diagnostics()
    cpt = lat.cells_per_thread
    staged = None if args.batch else bool(lat.tma_staging)
    lat.close()
    print(json.dumps({
        "case": f"{copies} x {args.side}x{args.side} {args.storage} variant {args.variant} "
                f"layer {args.width}" + (" (batched)" if args.batch else ""),
        "steps": args.steps, "cells_per_thread": cpt, "steps_per_launch": spl,
        "arithmetic": args.arithmetic,
        "tma_staging": staged,
        "mlups": cells / t / 1e6, "gbs": gbs,
        "frac_of_measured_hbm": gbs / peak if peak else None, "us_per_step": 1e6 * t / args.steps,
        "nonfinite_cells": d[5],
    }))


if __name__ == "__main__":
    main()
