"""Python binding of liblbm (include/lbm.h): argument marshalling only.

Every function named ``lbm_*`` here is the C entry point of the same name,
called through ctypes with raw pointers and sizes; the :class:`Lattice`
class wraps a handle for NumPy / PyTorch callers.  All arithmetic of the
time step runs in the CUDA library; there is no Python or CPU fallback, and
loading fails loudly if the library is missing.

PyTorch is used only for device memory (its caching allocator, through the
library's allocator hooks) and streams.
"""
from __future__ import annotations

import ctypes
import os
import warnings
from typing import Optional

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_WARN_UNSTABLE_PARAMS = 1
LBM_ERR_ARG = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_NONFINITE = -4
LBM_ERR_STATE = -5
LBM_ERR_TOO_LARGE = -6
LBM_VN_FIELDS = 15

STORAGE = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3}
VARIANT = {"none": 0, "I": 1, "II": 2, "III": 3, "viscous": 4}
BC = {"dirichlet": 0, "periodic": 1, "channel": 2}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
ARITHMETIC = {"native": 0, "compensated": 1}
ARITHMETIC_NAMES = {v: k for k, v in ARITHMETIC.items()}


class lbm_rates(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double * 9), ("n", ctypes.c_double), ("m", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lbm_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


_lib: Optional[ctypes.CDLL] = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64

# (name, restype, argtypes) of every entry point in include/lbm.h
SIGNATURES = [
    ("lbm_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.POINTER(lbm_rates),
                                  ctypes.c_int, _vp, ctypes.POINTER(lbm_allocator),
                                  ctypes.POINTER(_vp)]),
    ("lbm_set_sponge", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]),
    ("lbm_init_equilibrium", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
    ("lbm_step", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_moments", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
    ("lbm_diagnostics", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _vp]),
    ("lbm_state_bytes", ctypes.c_size_t, [_vp]),
    ("lbm_get_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int,
                                     ctypes.POINTER(_i64)]),
    ("lbm_set_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int, _i64]),
    ("lbm_time", _i64, [_vp]),
    ("lbm_set_stream", ctypes.c_int, [_vp, _vp]),
    ("lbm_set_source", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    ("lbm_set_launch_mode", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_set_cells_per_thread", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_cells_per_thread", ctypes.c_int, [_vp]),
    ("lbm_set_steps_per_launch", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_steps_per_launch", ctypes.c_int, [_vp]),
    ("lbm_set_arithmetic", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_probe_copy", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int, _vp]),
    ("lbm_get_arithmetic", ctypes.c_int, [_vp]),
    ("lbm_set_tma_staging", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_tma_staging", ctypes.c_int, [_vp]),
    ("lbm_destroy", None, [_vp]),
    ("lbm_last_error", ctypes.c_char_p, [_vp]),
    ("lbm_version", ctypes.c_char_p, []),
    ("lbm_diagnostics_noalloc", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp]),
    ("lbm_batch_instance_bytes", ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("lbm_lattice_bytes", ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int]),
    ("lbm_batch_create", ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(lbm_allocator),
                                        ctypes.POINTER(_vp)]),
    ("lbm_batch_set_tiling", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    ("lbm_batch_set_cells_per_thread", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_batch_cells_per_thread", ctypes.c_int, [_vp]),
    ("lbm_batch_set_steps_per_launch", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_batch_steps_per_launch", ctypes.c_int, [_vp]),
    ("lbm_batch_tma_staging", ctypes.c_int, [_vp]),
    ("lbm_batch_add", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.POINTER(lbm_rates),
                                     ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _i64,
                                     ctypes.POINTER(ctypes.c_int)]),
    ("lbm_batch_init_equilibrium", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int]),
    ("lbm_batch_init_pulse", ctypes.c_int, [_vp, ctypes.c_int] + [ctypes.c_double] * 4),
    ("lbm_init_pulse", ctypes.c_int, [_vp] + [ctypes.c_double] * 4),
    ("lbm_batch_step", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_batch_time", _i64, [_vp, ctypes.c_int]),
    ("lbm_batch_moments", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int]),
    ("lbm_batch_diagnostics", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, _vp]),
    ("lbm_batch_state_bytes", ctypes.c_size_t, [_vp, ctypes.c_int]),
    ("lbm_batch_get_state", ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]),
    ("lbm_batch_remove", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm_batch_count", ctypes.c_int, [_vp]),
    ("lbm_batch_set_stream", ctypes.c_int, [_vp, _vp]),
    ("lbm_batch_last_error", ctypes.c_char_p, [_vp]),
    ("lbm_batch_destroy", None, [_vp]),
    ("lbm_vn_growth", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                     _vp]),
    ("lbm_vn_chi_crit", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, _vp, _vp]),
    ("lbm_vn_last_error", ctypes.c_char_p, []),
    ("lbm3_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
     + [ctypes.c_double] * 4 + [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp,
                                 ctypes.POINTER(_vp)]),
    ("lbm3_set_sponge", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp] + [ctypes.c_double] * 4),
    ("lbm3_init_equilibrium", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("lbm3_step", ctypes.c_int, [_vp, ctypes.c_int]),
    ("lbm3_moments", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("lbm3_diagnostics", ctypes.c_int, [_vp] + [ctypes.c_int] * 6 + [_vp]),
    ("lbm3_state_bytes", ctypes.c_size_t, [_vp]),
    ("lbm3_get_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(_i64)]),
    ("lbm3_set_state", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _i64]),
    ("lbm3_time", _i64, [_vp]),
    ("lbm3_destroy", None, [_vp]),
    ("lbm3_last_error", ctypes.c_char_p, [_vp]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True) -> ctypes.CDLL:
    """Load liblbm.so (building it first if it is missing or stale and nvcc is
    available).  Raises if the library cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_stale and not _build.up_to_date():
        try:
            _build.build()
        except RuntimeError:
            if not os.path.exists(path):
                raise
    if not os.path.exists(path):
        raise RuntimeError(f"liblbm.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    """Raw address of a NumPy array or a torch tensor (None stays None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(type(x))


# ------------------------------------------------------ thin entry points ----

def lbm_version() -> str:
    return load().lbm_version().decode()


def lbm_last_error(h) -> str:
    return (load().lbm_last_error(h) or b"").decode()


def lbm_create(nx, ny, storage, rho0, ux0, uy0, rates: lbm_rates, bc, stream=None,
               alloc: Optional[lbm_allocator] = None):
    h = _vp()
    rc = load().lbm_create(int(nx), int(ny), int(storage), float(rho0), float(ux0), float(uy0),
                           ctypes.byref(rates), int(bc), stream,
                           ctypes.byref(alloc) if alloc is not None else None, ctypes.byref(h))
    return rc, h


def lbm_set_sponge(h, variant, chi_x_ptr, chi_y_ptr, rho_ref, ux_ref, uy_ref) -> int:
    return load().lbm_set_sponge(h, int(variant), chi_x_ptr, chi_y_ptr, float(rho_ref),
                                 float(ux_ref), float(uy_ref))


def lbm_init_equilibrium(h, rho_ptr, ux_ptr, uy_ptr, on_device) -> int:
    return load().lbm_init_equilibrium(h, rho_ptr, ux_ptr, uy_ptr, int(on_device))


def lbm_step(h, nsteps) -> int:
    return load().lbm_step(h, int(nsteps))


def lbm_moments(h, rho_ptr, ux_ptr, uy_ptr, on_device) -> int:
    return load().lbm_moments(h, rho_ptr, ux_ptr, uy_ptr, int(on_device))


def lbm_diagnostics(h, x0, y0, x1, y1, out_ptr) -> int:
    return load().lbm_diagnostics(h, int(x0), int(y0), int(x1), int(y1), out_ptr)


def lbm_state_bytes(h) -> int:
    return int(load().lbm_state_bytes(h))


def lbm_get_state(h, dst_ptr, nbytes, on_device):
    t = _i64()
    rc = load().lbm_get_state(h, dst_ptr, int(nbytes), int(on_device), ctypes.byref(t))
    return rc, t.value


def lbm_set_state(h, src_ptr, nbytes, on_device, time) -> int:
    return load().lbm_set_state(h, src_ptr, int(nbytes), int(on_device), int(time))


def lbm_time(h) -> int:
    return int(load().lbm_time(h))


def lbm_set_stream(h, stream) -> int:
    return load().lbm_set_stream(h, stream)


def lbm_set_source(h, amplitude, omega, phase) -> int:
    return load().lbm_set_source(h, float(amplitude), float(omega), float(phase))


LAUNCH_MODES = {"plain": 0, "pdl": 1, "graph": 2}


def lbm_set_launch_mode(h, mode) -> int:
    return load().lbm_set_launch_mode(h, int(mode))


def lbm_set_cells_per_thread(h, cells) -> int:
    return load().lbm_set_cells_per_thread(h, int(cells))


def lbm_cells_per_thread(h) -> int:
    return load().lbm_cells_per_thread(h)


def lbm_set_steps_per_launch(h, steps) -> int:
    return load().lbm_set_steps_per_launch(h, int(steps))


def lbm_steps_per_launch(h) -> int:
    return load().lbm_steps_per_launch(h)


def lbm_set_arithmetic(h, arithmetic) -> int:
    return load().lbm_set_arithmetic(h, int(arithmetic))


def lbm_get_arithmetic(h) -> int:
    return load().lbm_get_arithmetic(h)


def lbm_probe_copy(a_ptr, b_ptr, nbytes, iters, stream=None) -> int:
    return load().lbm_probe_copy(a_ptr, b_ptr, int(nbytes), int(iters), stream)


def lbm_set_tma_staging(h, on) -> int:
    return load().lbm_set_tma_staging(h, int(on))


def lbm_tma_staging(h) -> int:
    return load().lbm_tma_staging(h)


def lbm_destroy(h) -> None:
    load().lbm_destroy(h)


def lbm_diagnostics_noalloc(state_ptr, storage, nx, ny, bc, rho0, ux0, uy0, x0, y0, x1, y1,
                            out_ptr, out_on_device, stream=None) -> int:
    """Diagnostics of a caller-owned device population buffer with no device
    allocation (see include/lbm.h for who needs it and its limits)."""
    return load().lbm_diagnostics_noalloc(state_ptr, int(storage), int(nx), int(ny), int(bc),
                                          float(rho0), float(ux0), float(uy0), int(x0), int(y0),
                                          int(x1), int(y1), out_ptr, int(out_on_device), stream)


def lbm_vn_growth(variant_ptr, cases_ptr, ncases, nk, precision, growth_ptr, k_ptr,
                  stream=None) -> int:
    return load().lbm_vn_growth(variant_ptr, cases_ptr, int(ncases), int(nk), int(precision),
                                growth_ptr, k_ptr, stream)


def lbm_vn_chi_crit(variant_ptr, cases_ptr, ncases, nk, precision, chi_lo, chi_hi, nscan, iters,
                    tol, out_ptr, stream=None) -> int:
    return load().lbm_vn_chi_crit(variant_ptr, cases_ptr, int(ncases), int(nk), int(precision),
                                  float(chi_lo), float(chi_hi), int(nscan), int(iters),
                                  float(tol), out_ptr, stream)


def lbm_vn_last_error() -> str:
    return load().lbm_vn_last_error().decode()


def lbm3_create(nx, ny, nz, storage, rho0, u0, s15_ptr, n, m, bc, stream=None):
    h = _vp()
    rc = load().lbm3_create(int(nx), int(ny), int(nz), int(storage), float(rho0), float(u0[0]),
                            float(u0[1]), float(u0[2]), s15_ptr, float(n), float(m), int(bc),
                            stream, ctypes.byref(h))
    return rc, h


def lbm3_set_sponge(h, variant, cx_ptr, cy_ptr, cz_ptr, rho_ref, u_ref) -> int:
    return load().lbm3_set_sponge(h, int(variant), cx_ptr, cy_ptr, cz_ptr, float(rho_ref),
                                  float(u_ref[0]), float(u_ref[1]), float(u_ref[2]))


def lbm3_init_equilibrium(h, rho_ptr, ux_ptr, uy_ptr, uz_ptr) -> int:
    return load().lbm3_init_equilibrium(h, rho_ptr, ux_ptr, uy_ptr, uz_ptr)


def lbm3_step(h, nsteps) -> int:
    return load().lbm3_step(h, int(nsteps))


def lbm3_moments(h, rho_ptr, ux_ptr, uy_ptr, uz_ptr) -> int:
    return load().lbm3_moments(h, rho_ptr, ux_ptr, uy_ptr, uz_ptr)


def lbm3_diagnostics(h, x0, y0, z0, x1, y1, z1, out_ptr) -> int:
    return load().lbm3_diagnostics(h, int(x0), int(y0), int(z0), int(x1), int(y1), int(z1),
                                   out_ptr)


def lbm3_state_bytes(h) -> int:
    return load().lbm3_state_bytes(h)


def lbm3_get_state(h, dst_ptr, nbytes):
    t = _i64(0)
    rc = load().lbm3_get_state(h, dst_ptr, nbytes, ctypes.byref(t))
    return rc, t.value


def lbm3_set_state(h, src_ptr, nbytes, time) -> int:
    return load().lbm3_set_state(h, src_ptr, nbytes, int(time))


def lbm3_time(h) -> int:
    return load().lbm3_time(h)


def lbm3_destroy(h) -> None:
    load().lbm3_destroy(h)


def lbm3_last_error(h) -> str:
    return load().lbm3_last_error(h).decode()


def lbm_batch_instance_bytes(nx, ny, storage) -> int:
    return int(load().lbm_batch_instance_bytes(int(nx), int(ny), int(storage)))


def lbm_lattice_bytes(nx, ny, storage, bc, host_io) -> int:
    return int(load().lbm_lattice_bytes(int(nx), int(ny), int(storage), int(bc), int(host_io)))


def lbm_batch_create(storage, stream=None, alloc: Optional[lbm_allocator] = None):
    b = _vp()
    rc = load().lbm_batch_create(int(storage), stream,
                                 ctypes.byref(alloc) if alloc is not None else None,
                                 ctypes.byref(b))
    return rc, b


def lbm_batch_set_tiling(b, tile_x, tile_y) -> int:
    return load().lbm_batch_set_tiling(b, int(tile_x), int(tile_y))


def lbm_batch_set_cells_per_thread(b, cells) -> int:
    return load().lbm_batch_set_cells_per_thread(b, int(cells))


def lbm_batch_cells_per_thread(b) -> int:
    return load().lbm_batch_cells_per_thread(b)


def lbm_batch_set_steps_per_launch(b, steps) -> int:
    return load().lbm_batch_set_steps_per_launch(b, int(steps))


def lbm_batch_steps_per_launch(b) -> int:
    return load().lbm_batch_steps_per_launch(b)


def lbm_batch_tma_staging(b) -> int:
    return load().lbm_batch_tma_staging(b)


def lbm_batch_add(b, nx, ny, rho0, ux0, uy0, rates: lbm_rates, bc, variant, chi_x_ptr,
                  chi_y_ptr, rho_ref, ux_ref, uy_ref, nsteps):
    i = ctypes.c_int(-1)
    rc = load().lbm_batch_add(b, int(nx), int(ny), float(rho0), float(ux0), float(uy0),
                              ctypes.byref(rates), int(bc), int(variant), chi_x_ptr, chi_y_ptr,
                              float(rho_ref), float(ux_ref), float(uy_ref), int(nsteps),
                              ctypes.byref(i))
    return rc, i.value


def lbm_batch_init_equilibrium(b, i, rho_ptr, ux_ptr, uy_ptr, on_device) -> int:
    return load().lbm_batch_init_equilibrium(b, int(i), rho_ptr, ux_ptr, uy_ptr, int(on_device))


def lbm_batch_init_pulse(b, i, eps, half_width, x0, y0) -> int:
    return load().lbm_batch_init_pulse(b, int(i), float(eps), float(half_width), float(x0),
                                       float(y0))


def lbm_init_pulse(h, eps, half_width, x0, y0) -> int:
    return load().lbm_init_pulse(h, float(eps), float(half_width), float(x0), float(y0))


def lbm_batch_step(b, nsteps) -> int:
    return load().lbm_batch_step(b, int(nsteps))


def lbm_batch_time(b, i) -> int:
    return int(load().lbm_batch_time(b, int(i)))


def lbm_batch_moments(b, i, rho_ptr, ux_ptr, uy_ptr, on_device) -> int:
    return load().lbm_batch_moments(b, int(i), rho_ptr, ux_ptr, uy_ptr, int(on_device))


def lbm_batch_diagnostics(b, i, x0, y0, x1, y1, out_ptr) -> int:
    return load().lbm_batch_diagnostics(b, int(i), int(x0), int(y0), int(x1), int(y1), out_ptr)


def lbm_batch_state_bytes(b, i) -> int:
    return int(load().lbm_batch_state_bytes(b, int(i)))


def lbm_batch_get_state(b, i, dst_ptr, nbytes, on_device) -> int:
    return load().lbm_batch_get_state(b, int(i), dst_ptr, int(nbytes), int(on_device))


def lbm_batch_remove(b, i) -> int:
    return load().lbm_batch_remove(b, int(i))


def lbm_batch_count(b) -> int:
    return int(load().lbm_batch_count(b))


def lbm_batch_set_stream(b, stream) -> int:
    return load().lbm_batch_set_stream(b, stream)


def lbm_batch_last_error(b) -> str:
    return (load().lbm_batch_last_error(b) or b"").decode()


def lbm_batch_destroy(b) -> None:
    load().lbm_batch_destroy(b)


# ------------------------------------------------------------- helpers ----

def make_rates(s, n=0.5, m=0.5) -> lbm_rates:
    r = lbm_rates()
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), (9,))
    for k in range(9):
        r.s[k] = float(s[k])
    r.n, r.m = float(n), float(m)
    return r


class TorchAllocator:
    """Device memory from PyTorch's caching allocator, on a given stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self._torch = torch
        self.device = device
        self.stream = stream
        self._cb_alloc = ALLOC_FN(self._alloc)
        self._cb_free = FREE_FN(self._free)
        self.struct = lbm_allocator(self._cb_alloc, self._cb_free, None)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # the library turns NULL into LBM_ERR_OOM
            return None

    def _free(self, ptr, nbytes, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


def check(rc: int, h=None, what: str = "") -> int:
    if rc < 0:
        raise LbmError(rc, f"{what}: {lbm_last_error(h)}")
    if rc > 0:
        warnings.warn(f"liblbm warning {rc} in {what}: {lbm_last_error(h)}", RuntimeWarning,
                      stacklevel=3)
    return rc


class Lattice:
    """One lattice behind a liblbm handle.

    Host inputs/outputs are NumPy FP64 arrays; device ones are torch CUDA FP64
    tensors.  ``stream`` is a torch.cuda.Stream (default: the current stream).
    """

    def __init__(self, nx: int, ny: int, storage: str = "f32", rho0: float = 1.0,
                 u0=(0.0, 0.0), s=1.9, n: float = 0.5, m: float = 0.5, bc: str = "dirichlet",
                 stream=None, allocator: str = "torch", device: int = 0):
        import torch

        self.torch = torch
        torch.cuda.set_device(device)
        self.device = device
        self.nx, self.ny, self.storage, self.bc = int(nx), int(ny), storage, bc
        self.rho0, self.u0 = float(rho0), (float(u0[0]), float(u0[1]))
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = TorchAllocator(device, self.stream) if allocator == "torch" else None
        rc, h = lbm_create(nx, ny, STORAGE[storage], rho0, u0[0], u0[1], make_rates(s, n, m),
                           BC[bc], self.stream.cuda_stream,
                           self._alloc.struct if self._alloc else None)
        if rc < 0:
            raise LbmError(rc, lbm_last_error(None))
        self.h = h
        if rc > 0:
            warnings.warn(f"liblbm warning: {lbm_last_error(None)}", RuntimeWarning, stacklevel=2)

    @classmethod
    def from_workload(cls, w, storage: Optional[str] = None, init: str = "fields",
                      **kw) -> "Lattice":
        """Lattice for a workloads.Workload.  init="fields" uploads its initial
        fields; init="pulse" builds its Gaussian pulse on the device (workloads
        whose initial state is a pulse described by eps, b, x0, y0)."""
        lat = cls(w.nx, w.ny, storage or w.storage, w.rho0, w.u0, w.s, w.n, w.m, w.bc, **kw)
        try:
            lat.set_sponge(w.variant, w.chi_x, w.chi_y, w.rho_f, w.u_f)
            if w.bc == "channel":
                lat.set_source(*getattr(w, "source", (0.0, 0.0, 0.0)))
            if init == "pulse" and w.rho_dev is None:
                mt = w.meta
                lat.init_pulse(mt.get("eps", 0.0), mt.get("b", 1.0), mt.get("x0", 0.0),
                               mt.get("y0", 0.0))
            else:
                lat.init_equilibrium(*w.initial_fields())
        except Exception:
            lat.close()  # release the device memory of a lattice that failed set-up
            raise
        return lat

    @property
    def tma_staging(self) -> bool:
        """Whether two-step launches stage their input by TMA (Dirichlet; FP32, FP16 or BF16)."""
        return lbm_tma_staging(self.h) == 1

    @tma_staging.setter
    def tma_staging(self, on: bool) -> None:
        check(lbm_set_tma_staging(self.h, 1 if on else 0), self.h, "lbm_set_tma_staging")

    def set_source(self, amplitude: float, omega: float, phase: float = 0.0) -> None:
        """Line source of a channel lattice (Sec. 4.2): rho0 + amplitude
        sin(omega t + phase) on the left edge."""
        check(lbm_set_source(self.h, amplitude, omega, phase), self.h, "lbm_set_source")

    def set_stream(self, stream) -> None:
        """Issue later work on `stream` (a torch.cuda.Stream); the caller orders
        it after work already issued on the old one."""
        check(lbm_set_stream(self.h, stream.cuda_stream), self.h, "lbm_set_stream")
        self.stream = stream

    def init_pulse(self, eps: float, half_width: float, x0: float, y0: float) -> None:
        check(lbm_init_pulse(self.h, eps, half_width, x0, y0), self.h, "lbm_init_pulse")

    # ---- calls ----
    def set_sponge(self, variant: str, chi_x, chi_y, rho_ref: Optional[float] = None,
                   u_ref=None) -> int:
        cx = np.ascontiguousarray(chi_x, dtype=np.float64)
        cy = np.ascontiguousarray(chi_y, dtype=np.float64)
        assert cx.shape == (self.nx,) and cy.shape == (self.ny,)
        rho_ref = self.rho0 if rho_ref is None else rho_ref
        u_ref = self.u0 if u_ref is None else u_ref
        rc = lbm_set_sponge(self.h, VARIANT[variant], _ptr(cx), _ptr(cy), rho_ref, u_ref[0],
                            u_ref[1])
        return check(rc, self.h, "lbm_set_sponge")

    def init_equilibrium(self, rho, ux, uy) -> None:
        shp = (self.ny, self.nx)
        if isinstance(rho, np.ndarray):
            arrs = [np.ascontiguousarray(np.broadcast_to(a, shp), dtype=np.float64)
                    for a in (rho, ux, uy)]
            on_dev = 0
        else:
            arrs = [a.to(dtype=self.torch.float64).expand(shp).contiguous() for a in (rho, ux, uy)]
            assert all(a.is_cuda for a in arrs)
            on_dev = 1
        check(lbm_init_equilibrium(self.h, *(_ptr(a) for a in arrs), on_dev), self.h,
              "lbm_init_equilibrium")
        self._keep = arrs if on_dev else None

    def step(self, nsteps: int) -> None:
        check(lbm_step(self.h, nsteps), self.h, "lbm_step")

    def moments(self, device: bool = False):
        """(rho - rho0, u_x, u_y) at the current time, NumPy (host) or torch (device)."""
        shp = (self.ny, self.nx)
        if device:
            t = self.torch
            out = [t.empty(shp, dtype=t.float64, device=f"cuda:{self.device}") for _ in range(3)]
        else:
            out = [np.empty(shp) for _ in range(3)]
        check(lbm_moments(self.h, *(_ptr(a) for a in out), 1 if device else 0), self.h,
              "lbm_moments")
        return tuple(out)

    def diagnostics(self, region=None, raise_nonfinite: bool = False) -> np.ndarray:
        x0, y0, x1, y1 = region if region is not None else (0, 0, self.nx, self.ny)
        out = np.zeros(6)
        rc = lbm_diagnostics(self.h, x0, y0, x1, y1, _ptr(out))
        if rc == LBM_ERR_NONFINITE and not raise_nonfinite:
            return out
        check(rc, self.h, "lbm_diagnostics")
        return out

    def state_bytes(self) -> int:
        return lbm_state_bytes(self.h)

    def get_state(self):
        buf = np.empty(self.state_bytes(), dtype=np.uint8)
        rc, t = lbm_get_state(self.h, _ptr(buf), buf.nbytes, 0)
        check(rc, self.h, "lbm_get_state")
        return buf, t

    def set_state(self, buf: np.ndarray, time: int) -> None:
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lbm_set_state(self.h, _ptr(buf), buf.nbytes, 0, time), self.h, "lbm_set_state")

    @property
    def time(self) -> int:
        return lbm_time(self.h)

    @property
    def cells_per_thread(self) -> int:
        return lbm_cells_per_thread(self.h)

    @cells_per_thread.setter
    def cells_per_thread(self, cells: int) -> None:
        check(lbm_set_cells_per_thread(self.h, cells), self.h, "lbm_set_cells_per_thread")

    @property
    def arithmetic(self) -> str:
        """"native" (FP32 collision for FP32/16-bit storage, FP64 for FP64) or
        "compensated" (FP32 storage, float-float collision)."""
        rc = lbm_get_arithmetic(self.h)
        if rc < 0:  # a non-negative return is the mode, not a warning
            raise LbmError(rc, f"lbm_get_arithmetic: {lbm_last_error(self.h)}")
        return ARITHMETIC_NAMES[rc]

    @arithmetic.setter
    def arithmetic(self, name: str) -> None:
        check(lbm_set_arithmetic(self.h, ARITHMETIC[name]), self.h, "lbm_set_arithmetic")

    @property
    def steps_per_launch(self) -> int:
        return lbm_steps_per_launch(self.h)

    @steps_per_launch.setter
    def steps_per_launch(self, steps: int) -> None:
        check(lbm_set_steps_per_launch(self.h, steps), self.h, "lbm_set_steps_per_launch")

    def close(self) -> None:
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Lattice3:
    """One D3Q15 lattice behind an lbm3 handle (host FP64 fields [nz, ny, nx])."""

    def __init__(self, nx: int, ny: int, nz: int, storage: str = "f32", rho0: float = 1.0,
                 u0=(0.0, 0.0, 0.0), s=1.9, n: float = 0.5, m: float = 0.5,
                 bc: str = "dirichlet", stream=None, device: int = 0):
        import torch

        torch.cuda.set_device(device)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.rho0, self.u0 = float(rho0), tuple(float(v) for v in u0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        s15 = np.ascontiguousarray(np.broadcast_to(np.asarray(s, dtype=np.float64), (15,)))
        rc, h = lbm3_create(nx, ny, nz, STORAGE[storage], rho0, u0, s15.ctypes.data, n, m, BC[bc],
                            self.stream.cuda_stream)
        if rc < 0:
            raise LbmError(rc, lbm3_last_error(None))
        self.h = h
        if rc > 0:
            warnings.warn(f"liblbm warning: {lbm3_last_error(h)}", RuntimeWarning, stacklevel=2)

    def _check(self, rc: int, what: str) -> int:
        if rc < 0:
            raise LbmError(rc, f"{what}: {lbm3_last_error(self.h)}")
        if rc > 0:
            warnings.warn(f"liblbm warning in {what}: {lbm3_last_error(self.h)}", RuntimeWarning,
                          stacklevel=3)
        return rc

    def set_sponge(self, variant: str, chi_x, chi_y, chi_z, rho_ref=None, u_ref=None) -> int:
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (chi_x, chi_y, chi_z)]
        assert [a.shape for a in arrs] == [(self.nx,), (self.ny,), (self.nz,)]
        rho_ref = self.rho0 if rho_ref is None else rho_ref
        u_ref = self.u0 if u_ref is None else u_ref
        return self._check(lbm3_set_sponge(self.h, VARIANT[variant], *(a.ctypes.data for a in arrs),
                                           rho_ref, u_ref), "lbm3_set_sponge")

    def init_equilibrium(self, rho, ux, uy, uz) -> None:
        shp = (self.nz, self.ny, self.nx)
        arrs = [np.ascontiguousarray(np.broadcast_to(a, shp), dtype=np.float64)
                for a in (rho, ux, uy, uz)]
        self._check(lbm3_init_equilibrium(self.h, *(a.ctypes.data for a in arrs)),
                    "lbm3_init_equilibrium")

    def step(self, nsteps: int) -> None:
        self._check(lbm3_step(self.h, nsteps), "lbm3_step")

    def moments(self):
        shp = (self.nz, self.ny, self.nx)
        out = [np.empty(shp) for _ in range(4)]
        self._check(lbm3_moments(self.h, *(a.ctypes.data for a in out)), "lbm3_moments")
        return tuple(out)

    def diagnostics(self, region=None) -> np.ndarray:
        """FP64 sums over region (x0, y0, z0, x1, y1, z1) (default: all cells):
        sum rho', sum (j - rho0 u0) (3), acoustic energy, sum rho'^2, non-finite
        cells."""
        r = region if region is not None else (0, 0, 0, self.nx, self.ny, self.nz)
        out = np.zeros(7)
        rc = lbm3_diagnostics(self.h, *r, out.ctypes.data)
        if rc != LBM_ERR_NONFINITE:
            self._check(rc, "lbm3_diagnostics")
        return out

    def get_state(self):
        buf = np.empty(lbm3_state_bytes(self.h), dtype=np.uint8)
        rc, t = lbm3_get_state(self.h, buf.ctypes.data, buf.nbytes)
        self._check(rc, "lbm3_get_state")
        return buf, t

    def set_state(self, buf: np.ndarray, time: int) -> None:
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(lbm3_set_state(self.h, buf.ctypes.data, buf.nbytes, time), "lbm3_set_state")

    @property
    def time(self) -> int:
        return lbm3_time(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            lbm3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
