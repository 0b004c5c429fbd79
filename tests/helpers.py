"""Shared helpers of the test suite: run one workload on the oracle or on the
CUDA library and compare fields."""
from __future__ import annotations

import numpy as np


def oracle_problem(core, w):
    return core.Problem(w.nx, w.ny, w.s, n=w.n, m=w.m, variant=w.variant, bc=w.bc, rho0=w.rho0,
                        u0=w.u0, rho_f=w.rho_f, u_f=w.u_f, chi_x=w.chi_x, chi_y=w.chi_y,
                        src_amp=w.source[0], src_omega=w.source[1], src_phase=w.source[2])


def run_oracle(w, steps=None, nthreads=0):
    """Oracle fields (rho', ux, uy) of workload w after `steps` (default w.steps)."""
    from oracle import core

    st = core.State(oracle_problem(core, w), *w.initial_fields())
    st.run(w.steps if steps is None else steps, nthreads)
    return st.moments()


def run_gpu(w, storage=None, steps=None):
    """CUDA-library fields (rho', ux, uy) of workload w after `steps`.  storage
    "f32c": FP32 storage with the compensated (float-float) collision."""
    from paper_1203_6350_gb300 import lbm

    storage = storage or w.storage
    comp = storage == "f32c"
    with lbm.Lattice.from_workload(w, storage="f32" if comp else storage) as lat:
        if comp:
            lat.arithmetic = "compensated"
        lat.step(w.steps if steps is None else steps)
        return lat.moments()


def rel_l2(a, b) -> float:
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def ring_regions(nx, ny, r=2):
    """The outermost r cells of an nx x ny lattice as four disjoint rectangles
    (x0, y0, x1, y1): the cells next to the Dirichlet wall, behind the layer."""
    return [(0, 0, nx, r), (0, ny - r, nx, ny), (0, r, r, ny - r), (nx - r, r, nx, ny - r)]


def interior_region(w):
    """The cells with chi = 0 of a workload with a `width`-cell layer on every side."""
    return (w.width, w.width, w.nx - w.width, w.ny - w.width)
