"""Von Neumann stability maps on the GPU (lbm_vn_* in include/lbm.h).

Argument marshalling only: the linearisation, the eigenvalue problems and the
scan-and-bisection for the critical damping strength run in liblbm.  A case
is (rates s[9], Guo weights n and m, target velocity u^f, wave direction
theta, damping strength chi) with a damping variant; see Secs. 3.2-3.3.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import lbm

FIELDS = ("s0", "s1", "s2", "s3", "s4", "s5", "s6", "s7", "s8", "n", "m", "ux_f", "uy_f",
          "theta", "chi")
VARIANTS = ("none", "I", "II", "III")
PRECISION = {"f64": lbm.STORAGE["f64"], "f32": lbm.STORAGE["f32"]}


def case(s, chi: float = 0.0, n: float = 0.5, m: float = 0.5, u_f=(0.0, 0.0),
         theta: float = 0.0) -> np.ndarray:
    """One case record; s is one rate (all nine equal) or nine rates."""
    s9 = np.broadcast_to(np.asarray(s, dtype=np.float64), (9,))
    return np.concatenate([s9, [n, m, u_f[0], u_f[1], theta, chi]]).astype(np.float64)


def _marshal(variants: Sequence, cases):
    c = np.ascontiguousarray(np.atleast_2d(np.asarray(cases, dtype=np.float64)))
    if c.shape[1] != lbm.LBM_VN_FIELDS:
        raise ValueError(f"a case has {lbm.LBM_VN_FIELDS} fields, got {c.shape[1]}")
    if isinstance(variants, str):
        variants = [variants] * c.shape[0]
    v = np.ascontiguousarray([VARIANTS.index(x) if isinstance(x, str) else int(x)
                              for x in variants], dtype=np.int32)
    if v.shape[0] != c.shape[0]:
        raise ValueError("one variant per case")
    return v, c


def _stream(stream):
    if stream is not None:
        return stream.cuda_stream
    import torch

    return torch.cuda.current_stream().cuda_stream


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise lbm.LbmError(rc, f"{what}: {lbm.lbm_vn_last_error()}")


def growth(variants, cases, nk: int = 400, precision: str = "f32", stream=None):
    """(growth[c], |k| at the maximum) for each case."""
    v, c = _marshal(variants, cases)
    g = np.empty(c.shape[0])
    k = np.empty(c.shape[0])
    _check(lbm.lbm_vn_growth(v.ctypes.data, c.ctypes.data, c.shape[0], nk, PRECISION[precision],
                             g.ctypes.data, k.ctypes.data, _stream(stream)), "lbm_vn_growth")
    return g, k


def chi_crit(variants, cases, nk: int = 400, precision: str = "f32", chi_lo: float = 0.0,
             chi_hi: float = 8.0, nscan: int = 17, iters: int = 40,
             tol: Optional[float] = None, stream=None) -> np.ndarray:
    """Critical damping strength of each case (the chi field is ignored);
    tol defaults to 1e-9 (FP64) or 1e-5 (FP32)."""
    v, c = _marshal(variants, cases)
    tol = (1e-9 if precision == "f64" else 1e-5) if tol is None else tol
    out = np.empty(c.shape[0])
    _check(lbm.lbm_vn_chi_crit(v.ctypes.data, c.ctypes.data, c.shape[0], nk,
                               PRECISION[precision], chi_lo, chi_hi, nscan, iters, tol,
                               out.ctypes.data, _stream(stream)), "lbm_vn_chi_crit")
    return out
