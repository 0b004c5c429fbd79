"""GB300-native (sm_103a) time step of the D2Q9 MRT lattice Boltzmann scheme with
the absorbing-layer damping terms of Xu & Sagaut (arXiv:1203.6350).

The compute lives in ``liblbm.so`` (CUDA, built from ``csrc/`` by
:mod:`paper_1203_6350_gb300.build`); :mod:`paper_1203_6350_gb300.lbm` is its
ctypes binding.  Importing this package does not load the library; the first
call does, and fails loudly if it is missing.
"""
from . import build  # noqa: F401

__all__ = ["build", "lbm"]
