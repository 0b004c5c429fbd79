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
    """CUDA-library fields (rho', ux, uy) of workload w after `steps`."""
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice.from_workload(w, storage=storage) as lat:
        lat.step(w.steps if steps is None else steps)
        return lat.moments()


def rel_l2(a, b) -> float:
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
