"""FP64 CPU oracle for the D2Q9 MRT lattice Boltzmann step with absorbing layers.

TEST INFRASTRUCTURE.  Everything in this package exists to check the CUDA path
and is never called by it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it.

Contents
--------
``lbm_oracle.c`` / :mod:`oracle.core`
    Plain C, FP64, population-space step (OpenMP over rows) and its ctypes
    loader.  Follows Xu & Sagaut (arXiv:1203.6350) Sec. 2, Eqs. (blbs),
    (blbs-abc-1), (app:newbgka), (app:newbgka2), (app:bgk_no2ordor2), App. A.1.
:mod:`oracle.twin`
    The same definition written again with NumPy, for brute-force cross-checks
    of the C code on tiny lattices.
:mod:`oracle.vonneumann`
    Linearised scheme and Von Neumann amplification matrix (Sec. 3.2,
    Eqs. (eq:linearized), (perturb-w-f), (sec:matrix)), from an analytic
    Jacobian.
:mod:`oracle.pulse`
    Closed-form 2-D acoustic Gaussian pulse (Sec. 4.1, Bessel integral).
:mod:`oracle.diagnostics`
    FP64 reductions over oracle fields (mass, momentum, acoustic energy,
    E_L2 of Sec. 4.1).
"""
