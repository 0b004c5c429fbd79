"""ctypes loader and build step for the C oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE: see the package docstring.  Parity status: pinned by
``tests/test_oracle_pins.py`` (conservation, k = 0 closed forms, Von Neumann
plane waves, acoustic pulse, symmetry, NumPy twin).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")

VARIANTS = {"none": 0, "I": 1, "II": 2, "III": 3, "viscous": 4}
BCS = {"dirichlet": 0, "periodic": 1, "channel": 2}


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("bc", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("rho0", ctypes.c_double),
        ("ux0", ctypes.c_double),
        ("uy0", ctypes.c_double),
        ("rho_f", ctypes.c_double),
        ("ux_f", ctypes.c_double),
        ("uy_f", ctypes.c_double),
        ("s", ctypes.c_double * 9),
        ("n", ctypes.c_double),
        ("m", ctypes.c_double),
        ("src_amp", ctypes.c_double),
        ("src_omega", ctypes.c_double),
        ("src_phase", ctypes.c_double),
        ("t0", ctypes.c_double),
    ]


def build(force: bool = False, quiet: bool = True) -> str:
    """Compile ``lbm_oracle.c`` into ``oracle/_build/liblbm_oracle.so`` (gcc, -O2,
    OpenMP when the compiler supports it).  Returns the library path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = tempfile.NamedTemporaryFile(dir=_BUILD, suffix=".so", delete=False).name
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    for extra in (["-fopenmp"], []):
        cmd = base[:1] + extra + base[1:]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _LIB)
            return _LIB
        if not quiet:
            sys.stderr.write(r.stderr)
    raise RuntimeError("could not compile the oracle: " + r.stderr)


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        _lib.oracle_init.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_run.argtypes = [pp, dp, dp, dp, ctypes.c_int, ctypes.c_int]
        _lib.oracle_moments.argtypes = [pp, dp, dp, dp, dp]
        _lib.oracle_lambda.argtypes = [dp, dp]
        _lib.oracle_feq.argtypes = [ctypes.c_double] * 3 + [dp]
        _lib.oracle_feq_linear.argtypes = [ctypes.c_double] * 3 + [dp]
        _lib.oracle_collide_cell.argtypes = [pp, dp, ctypes.c_double, dp, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.oracle_tables.argtypes = [ip, ip, dp, dp]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """Statement of one lattice problem in the paper's terms.

    ``s`` are the nine rates of S in the row order of M (App. A.1); ``s[0:3]``
    act on the conserved rows (rate s_c), ``n``/``m`` are the Guo weights,
    ``rho0/u0`` the far-field (boundary) state, ``rho_f/u_f`` the reference
    state q_ref of the absorbing term, ``chi_x``/``chi_y`` the per-axis
    absorbing strengths (chi = max of the two at a cell).  With bc="channel"
    (the line source of Sec. 4.2) the left edge is a source of density
    rho0 + src_amp sin(src_omega t + src_phase) moving at u0, the right edge an
    outflow, and y is periodic.
    """

    nx: int
    ny: int
    s: np.ndarray
    n: float = 0.5
    m: float = 0.5
    variant: str = "II"
    bc: str = "dirichlet"
    rho0: float = 1.0
    u0: tuple = (0.0, 0.0)
    rho_f: float = 1.0
    u_f: tuple = (0.0, 0.0)
    chi_x: np.ndarray = field(default=None)
    chi_y: np.ndarray = field(default=None)
    src_amp: float = 0.0
    src_omega: float = 0.0
    src_phase: float = 0.0

    def __post_init__(self):
        self.s = np.asarray(self.s, dtype=np.float64)
        if self.chi_x is None:
            self.chi_x = np.zeros(self.nx)
        if self.chi_y is None:
            self.chi_y = np.zeros(self.ny)
        self.chi_x = np.ascontiguousarray(self.chi_x, dtype=np.float64)
        self.chi_y = np.ascontiguousarray(self.chi_y, dtype=np.float64)

    def params(self) -> _Params:
        p = _Params()
        p.nx, p.ny = self.nx, self.ny
        p.bc = BCS[self.bc]
        p.variant = VARIANTS[self.variant]
        p.rho0, (p.ux0, p.uy0) = self.rho0, self.u0
        p.rho_f, (p.ux_f, p.uy_f) = self.rho_f, self.u_f
        for k in range(9):
            p.s[k] = float(self.s[k])
        p.n, p.m = self.n, self.m
        p.src_amp, p.src_omega, p.src_phase = self.src_amp, self.src_omega, self.src_phase
        p.t0 = 0.0
        return p


class State:
    """Populations f[9, ny, nx] (FP64, full values, not deviations) of one
    problem, advanced by the C oracle."""

    def __init__(self, prob: Problem, rho: np.ndarray, ux: np.ndarray, uy: np.ndarray):
        self.prob = prob
        self._p = prob.params()
        self.f = np.zeros((9, prob.ny, prob.nx))
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        ux = np.ascontiguousarray(np.broadcast_to(ux, rho.shape), dtype=np.float64)
        uy = np.ascontiguousarray(np.broadcast_to(uy, rho.shape), dtype=np.float64)
        rc = lib().oracle_init(ctypes.byref(self._p), _dp(rho), _dp(ux), _dp(uy), _dp(self.f))
        if rc != 0:
            raise ValueError(f"oracle_init failed ({rc})")
        self.t = 0

    def run(self, nsteps: int, nthreads: int = 0) -> "State":
        self._p.t0 = float(self.t)
        rc = lib().oracle_run(ctypes.byref(self._p), _dp(self.prob.chi_x), _dp(self.prob.chi_y),
                              _dp(self.f), int(nsteps), int(nthreads))
        if rc != 0:
            raise RuntimeError(f"oracle_run failed ({rc})")
        self.t += nsteps
        return self

    def moments(self):
        """(rho - rho0, u_x, u_y), each [ny, nx] FP64."""
        shp = (self.prob.ny, self.prob.nx)
        r, ux, uy = np.empty(shp), np.empty(shp), np.empty(shp)
        lib().oracle_moments(ctypes.byref(self._p), _dp(self.f), _dp(r), _dp(ux), _dp(uy))
        return r, ux, uy


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.empty(9)
    lib().oracle_feq(rho, ux, uy, _dp(out))
    return out


def feq_linear(rho: float, jx: float, jy: float) -> np.ndarray:
    out = np.empty(9)
    lib().oracle_feq_linear(rho, jx, jy, _dp(out))
    return out


def lambda_matrix(s) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty(81)
    if lib().oracle_lambda(_dp(s), _dp(out)) != 0:
        raise RuntimeError("singular M")
    return out.reshape(9, 9)


def collide_cell(prob: Problem, chi: float, f: np.ndarray) -> np.ndarray:
    p = prob.params()
    lam = np.ascontiguousarray(lambda_matrix(prob.s).ravel())
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(9)
    lib().oracle_collide_cell(ctypes.byref(p), _dp(lam), float(chi), _dp(f), _dp(out))
    return out


def tables():
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = np.empty(9)
    mm = np.empty(81)
    lib().oracle_tables(cx, cy, _dp(w), _dp(mm))
    return np.array(cx[:]), np.array(cy[:]), w, mm.reshape(9, 9)


def omp_threads() -> int:
    """Threads the oracle uses by default (OpenMP's default, else 1)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
