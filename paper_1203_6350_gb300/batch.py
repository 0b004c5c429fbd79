"""Python wrapper of the batched C ABI (lbm_batch_* in include/lbm.h).

Argument marshalling only: every step of the path runs in liblbm.  A
:class:`Batch` holds many independent lattices of one storage type and
advances all active ones with one persistent launch per time step.
"""
from __future__ import annotations

import warnings
from typing import Optional

import numpy as np

from . import lbm


class Batch:
    def __init__(self, storage: str = "f32", stream=None, allocator: str = "torch",
                 device: int = 0, tiling: Optional[tuple] = None, config: Optional[dict] = None):
        """config: a kernel configuration {"cells", "steps_per_launch", "tile"}
        (as autotune.tuned_config returns); tiling: a tile shape only."""
        import torch

        self.torch = torch
        torch.cuda.set_device(device)
        self.device = device
        self.storage = storage
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = lbm.TorchAllocator(device, self.stream) if allocator == "torch" else None
        rc, b = lbm.lbm_batch_create(lbm.STORAGE[storage], self.stream.cuda_stream,
                                     self._alloc.struct if self._alloc else None)
        if rc != 0:
            raise lbm.LbmError(rc, "lbm_batch_create failed")
        self.b = b
        self.shapes = {}
        if tiling is not None:
            self.set_tiling(*tiling)
        if config is not None:
            self.configure(config["cells"], config["steps_per_launch"], config["tile"])

    def _check(self, rc: int, what: str) -> int:
        if rc < 0:
            raise lbm.LbmError(rc, f"{what}: {lbm.lbm_batch_last_error(self.b)}")
        if rc > 0:
            warnings.warn(f"liblbm warning {rc} in {what}", RuntimeWarning, stacklevel=3)
        return rc

    def set_stream(self, stream) -> None:
        """Issue later work on `stream` (a torch.cuda.Stream); the caller orders
        it after work already issued on the old one."""
        self._check(lbm.lbm_batch_set_stream(self.b, stream.cuda_stream), "lbm_batch_set_stream")
        self.stream = stream

    def set_tiling(self, tile_x: int, tile_y: int) -> None:
        self._check(lbm.lbm_batch_set_tiling(self.b, tile_x, tile_y), "lbm_batch_set_tiling")

    def configure(self, cells: int, steps_per_launch: int, tile) -> None:
        """Kernel (cells per thread, time steps per launch) and one-step tile shape."""
        if steps_per_launch == 1:
            self.steps_per_launch = 1
        self.cells_per_thread = cells
        self.steps_per_launch = steps_per_launch
        self.set_tiling(*tile)

    @property
    def cells_per_thread(self) -> int:
        return lbm.lbm_batch_cells_per_thread(self.b)

    @cells_per_thread.setter
    def cells_per_thread(self, cells: int) -> None:
        self._check(lbm.lbm_batch_set_cells_per_thread(self.b, cells),
                    "lbm_batch_set_cells_per_thread")

    @property
    def steps_per_launch(self) -> int:
        return lbm.lbm_batch_steps_per_launch(self.b)

    @steps_per_launch.setter
    def steps_per_launch(self, steps: int) -> None:
        self._check(lbm.lbm_batch_set_steps_per_launch(self.b, steps),
                    "lbm_batch_set_steps_per_launch")

    def add(self, nx, ny, steps, s=1.9, n=0.5, m=0.5, rho0=1.0, u0=(0.0, 0.0), bc="dirichlet",
            variant="none", chi_x=None, chi_y=None, rho_ref=None, u_ref=None) -> int:
        cx = np.ascontiguousarray(np.zeros(nx) if chi_x is None else chi_x, dtype=np.float64)
        cy = np.ascontiguousarray(np.zeros(ny) if chi_y is None else chi_y, dtype=np.float64)
        rho_ref = rho0 if rho_ref is None else rho_ref
        u_ref = u0 if u_ref is None else u_ref
        rc, i = lbm.lbm_batch_add(self.b, nx, ny, rho0, u0[0], u0[1], lbm.make_rates(s, n, m),
                                  lbm.BC[bc], lbm.VARIANT[variant], cx.ctypes.data,
                                  cy.ctypes.data, rho_ref, u_ref[0], u_ref[1], steps)
        self._check(rc, "lbm_batch_add")
        self.shapes[i] = (ny, nx)
        return i

    def add_workload(self, w, steps: Optional[int] = None, init="fields") -> int:
        """Add a workloads.Workload (its own storage field is ignored: the batch's
        storage applies).  init="fields" uploads its initial fields, "pulse"
        builds its Gaussian pulse on the device, None leaves it uninitialised."""
        i = self.add(w.nx, w.ny, w.steps if steps is None else steps, w.s, w.n, w.m, w.rho0,
                     w.u0, w.bc, w.variant, w.chi_x, w.chi_y, w.rho_f, w.u_f)
        try:
            if init == "pulse" and w.rho_dev is None:
                mt = w.meta
                self.init_pulse(i, mt.get("eps", 0.0), mt.get("b", 1.0), mt.get("x0", 0.0),
                                mt.get("y0", 0.0))
            elif init:
                self.init_equilibrium(i, *w.initial_fields())
        except Exception:
            self.remove(i)  # no half-initialised instance stays in the batch
            raise
        return i

    def init_pulse(self, i, eps, half_width, x0, y0) -> None:
        self._check(lbm.lbm_batch_init_pulse(self.b, i, eps, half_width, x0, y0),
                    "lbm_batch_init_pulse")

    def init_equilibrium(self, i, rho, ux, uy) -> None:
        shp = self.shapes[i]
        if isinstance(rho, np.ndarray):
            arrs = [np.ascontiguousarray(np.broadcast_to(a, shp), dtype=np.float64)
                    for a in (rho, ux, uy)]
            on_dev = 0
        else:
            arrs = [a.to(dtype=self.torch.float64).expand(shp).contiguous() for a in (rho, ux, uy)]
            on_dev = 1
        self._check(lbm.lbm_batch_init_equilibrium(self.b, i, *(lbm._ptr(a) for a in arrs), on_dev),
                    "lbm_batch_init_equilibrium")
        self._keep = arrs if on_dev else None

    def step(self, nsteps: int) -> None:
        self._check(lbm.lbm_batch_step(self.b, nsteps), "lbm_batch_step")

    def time(self, i) -> int:
        return lbm.lbm_batch_time(self.b, i)

    def moments(self, i):
        shp = self.shapes[i]
        out = [np.empty(shp) for _ in range(3)]
        self._check(lbm.lbm_batch_moments(self.b, i, *(a.ctypes.data for a in out), 0),
                    "lbm_batch_moments")
        return tuple(out)

    def diagnostics(self, i, region=None) -> np.ndarray:
        ny, nx = self.shapes[i]
        x0, y0, x1, y1 = region if region is not None else (0, 0, nx, ny)
        out = np.zeros(6)
        rc = lbm.lbm_batch_diagnostics(self.b, i, x0, y0, x1, y1, out.ctypes.data)
        if rc != lbm.LBM_ERR_NONFINITE:
            self._check(rc, "lbm_batch_diagnostics")
        return out

    def get_state(self, i) -> np.ndarray:
        """Raw population buffer of instance i (layout of Lattice.get_state)."""
        buf = np.empty(lbm.lbm_batch_state_bytes(self.b, i), dtype=np.uint8)
        self._check(lbm.lbm_batch_get_state(self.b, i, buf.ctypes.data, buf.nbytes, 0),
                    "lbm_batch_get_state")
        return buf

    def remove(self, i) -> None:
        self._check(lbm.lbm_batch_remove(self.b, i), "lbm_batch_remove")
        self.shapes.pop(i, None)

    def __len__(self) -> int:
        return lbm.lbm_batch_count(self.b)

    def close(self) -> None:
        if getattr(self, "b", None):
            lbm.lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
