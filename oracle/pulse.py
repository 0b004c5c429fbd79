"""Closed-form 2-D acoustic Gaussian pulse (Sec. 4.1).

TEST INFRASTRUCTURE (see the package docstring).

Initial density rho0 + eps exp(-alpha r^2), alpha = ln 2 / b^2, zero velocity
perturbation on a uniform mean flow U0 e_x (Eqs. pulseprofile, 3:para0).  In
the inviscid linear limit the density perturbation is the Hankel-transform
integral of Sec. 4.1:

    rho'(x, t) = eps / (2 alpha) * int_0^inf exp(-xi^2 / (4 alpha))
                 cos(c_s t xi) J0(xi eta) xi d xi,
    eta = |x - x0 - U0 t e_x|.

At t = 0 the integral is eps exp(-alpha eta^2) exactly (Hankel transform of a
Gaussian), which is one of the pins of this module.  The integral is evaluated
with Gauss-Legendre quadrature on [0, xi_max], xi_max chosen so that the
Gaussian factor has fallen below exp(-60).
"""
from __future__ import annotations

import numpy as np
from scipy.special import j0, roots_legendre

CS = 1.0 / np.sqrt(3.0)


def rho_prime(x, y, t, eps=1e-3, b=3.0, x0=0.0, y0=0.0, U0=0.0, cs=CS, nquad=4000):
    alpha = np.log(2.0) / b**2
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    eta = np.sqrt((x - x0 - U0 * t) ** 2 + (y - y0) ** 2)
    ximax = np.sqrt(4.0 * alpha * 60.0)
    z, w = roots_legendre(nquad)
    xi = 0.5 * ximax * (z + 1.0)
    w = 0.5 * ximax * w
    g = np.exp(-xi**2 / (4 * alpha)) * np.cos(cs * t * xi) * xi * w  # [nquad]
    flat = eta.ravel()
    out = np.empty_like(flat)
    chunk = 4096
    for a in range(0, flat.size, chunk):
        e = flat[a : a + chunk]
        out[a : a + chunk] = j0(np.outer(e, xi)) @ g
    return (eps / (2 * alpha) * out).reshape(eta.shape)
