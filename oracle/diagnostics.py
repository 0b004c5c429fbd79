"""FP64 reductions over oracle fields.

TEST INFRASTRUCTURE (see the package docstring).

Over a rectangle [x0, x1) x [y0, y1) of a state with fields rho' = rho - rho0
and u:
  0: sum rho'                                   (mass deviation)
  1: sum (rho u_x - rho0 u0x)                   (momentum deviation, x)
  2: sum (rho u_y - rho0 u0y)                   (momentum deviation, y)
  3: sum [c_s^2 rho'^2 / (2 rho0) + rho0 |u - u0|^2 / 2]   (acoustic energy)
  4: sum rho'^2                                 (numerator of E_L2, Sec. 4.1,
                                                 with rho_ref = rho0)
  5: number of cells whose rho' or u is not finite
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0


def reduce_fields(rho_dev, ux, uy, rho0=1.0, u0=(0.0, 0.0), region=None) -> np.ndarray:
    ny, nx = rho_dev.shape
    x0, y0, x1, y1 = region if region is not None else (0, 0, nx, ny)
    r = rho_dev[y0:y1, x0:x1]
    vx = ux[y0:y1, x0:x1]
    vy = uy[y0:y1, x0:x1]
    rho = rho0 + r
    out = np.zeros(6)
    out[0] = r.sum()
    out[1] = (rho * vx - rho0 * u0[0]).sum()
    out[2] = (rho * vy - rho0 * u0[1]).sum()
    out[3] = (CS2 * r**2 / (2 * rho0) + rho0 * ((vx - u0[0]) ** 2 + (vy - u0[1]) ** 2) / 2).sum()
    out[4] = (r**2).sum()
    out[5] = float((~(np.isfinite(r) & np.isfinite(vx) & np.isfinite(vy))).sum())
    return out


def e_l2(rho_dev, rho0=1.0) -> float:
    """E_L2 of Sec. 4.1 with rho_ref = rho0 everywhere."""
    return float(np.sqrt((rho_dev**2).sum() / (rho_dev.size * rho0**2)))
