"""NumPy restatement of the oracle step, for brute-force checks of the C code on
tiny lattices.

TEST INFRASTRUCTURE (see the package docstring).  This is the same definition
as ``lbm_oracle.c`` -- Eq. (blbs-abc-1) with Gamma = chi I and the three
damping variants of Secs. 2.2.1-2.2.3 -- written a second time, vectorised over
cells, with Lambda = M^{-1} S M taken from ``numpy.linalg.inv``.  It is meant to
catch indexing and streaming mistakes in the C code; the physics pins in
``tests/test_oracle_pins.py`` catch mistakes of definition.
"""
from __future__ import annotations

import numpy as np

# App. A.1: the D2Q9 transformation matrix, and the velocity set read off its rows 1-2.
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)
C = M[1:3].T.astype(int)  # c_i = (M[1,i], M[2,i])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq(rho, ux, uy):
    """f^eq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u); arrays broadcast, axis 0 = i."""
    rho, ux, uy = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, ux, uy)))
    cu = C[:, 0].reshape((9,) + (1,) * rho.ndim) * ux + C[:, 1].reshape((9,) + (1,) * rho.ndim) * uy
    w = W.reshape((9,) + (1,) * rho.ndim)
    return w * rho * (1 + 3 * cu + 4.5 * cu**2 - 1.5 * (ux**2 + uy**2))


def feq_linear(rho, jx, jy):
    rho, jx, jy = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, jx, jy)))
    sh = (9,) + (1,) * rho.ndim
    return W.reshape(sh) * (rho + 3 * (C[:, 0].reshape(sh) * jx + C[:, 1].reshape(sh) * jy))


def source_rho(source, rho0, t):
    """Density of the line source (channel boundary) at time t."""
    amp, omega, phase = source
    return rho0 + amp * np.sin(omega * t + phase)


def init(rho, ux, uy, bc="dirichlet", rho0=1.0, u0=(0.0, 0.0), source=(0.0, 0.0, 0.0)):
    """f = f^eq(rho, u); with the Dirichlet rule, populations entering from
    outside take f^eq(rho0, u0).  Channel: those entering at the left edge take
    the source equilibrium of time -1, those entering at the right edge the
    equilibrium of the column inside (x = nx - 2) in the same row."""
    rho, ux, uy = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, ux, uy)))
    f = feq(rho, ux, uy)
    if bc == "dirichlet":
        _apply_dirichlet(f, feq(rho0, *u0))
    elif bc == "channel":
        fs = feq(source_rho(source, rho0, -1.0), *u0)
        fo = feq(rho[:, -2], ux[:, -2], uy[:, -2])  # [9, ny]
        for i in range(9):
            if C[i, 0] == 1:
                f[i, :, 0] = fs[i]
            elif C[i, 0] == -1:
                f[i, :, -1] = fo[i]
    return f


def _apply_dirichlet(f, fb):
    _, ny, nx = f.shape
    for i in range(9):
        cx, cy = C[i]
        for iy in range(ny):
            for ix in range(nx):
                sx, sy = ix - cx, iy - cy
                if not (0 <= sx < nx and 0 <= sy < ny):
                    f[i, iy, ix] = fb[i]


def step(f, chi, s, variant="II", n=0.5, m=0.5, rho_f=1.0, u_f=(0.0, 0.0), bc="dirichlet",
         rho0=1.0, u0=(0.0, 0.0), source=(0.0, 0.0, 0.0), t=0):
    """One time step of the scheme from time t.  f: [9, ny, nx]; chi: [ny, nx]."""
    kw = dict(source=source, t=t)
    lam = np.linalg.inv(M) @ np.diag(s) @ M
    if variant == "viscous":
        # Sec. 4.1 comparison: no damping term, the non-conserved rates fall
        # linearly to 1 across the layer; chi carries the layer fraction r.
        r = chi
        rho = f.sum(0)
        jx = np.tensordot(C[:, 0], f, 1)
        jy = np.tensordot(C[:, 1], f, 1)
        fs = feq(rho, jx / rho, jy / rho)
        out_post = np.empty_like(f)
        minv = np.linalg.inv(M)
        for iy in range(f.shape[1]):
            for ix in range(f.shape[2]):
                sk = np.array(s, dtype=np.float64)
                sk[3:] = sk[3:] + (1.0 - sk[3:]) * r[iy, ix]
                lam_c = minv @ np.diag(sk) @ M
                out_post[:, iy, ix] = f[:, iy, ix] + lam_c @ (fs[:, iy, ix] - f[:, iy, ix])
        return _stream(out_post, bc, rho0, u0, **kw)
    if variant == "none":  # no absorbing term: F = 0, so rho* = rho and j* = j
        chi = np.zeros_like(chi)
    rho = f.sum(0)
    jx = np.tensordot(C[:, 0], f, 1)
    jy = np.tensordot(C[:, 1], f, 1)
    jfx, jfy = rho_f * u_f[0], rho_f * u_f[1]
    rs = (rho + n * chi * rho_f) / (1 + n * chi)
    jxs = (jx + m * chi * jfx) / (1 + m * chi)
    jys = (jy + m * chi * jfy) / (1 + m * chi)
    fs = feq(rs, jxs / rs, jys / rs)
    coll = np.tensordot(lam, fs - f, 1)
    if variant == "I":
        t = chi * (feq(rho_f, *u_f)[:, None, None] - f)
    elif variant == "II":
        t = chi * (feq(rho_f, *u_f)[:, None, None] - fs)
    elif variant == "III":
        t = chi * (feq_linear(rho_f, jfx, jfy)[:, None, None] - feq_linear(rs, jxs, jys))
    else:
        t = 0.0
    post = f + coll + t
    return _stream(post, bc, rho0, u0, **kw)


def _stream(post, bc, rho0, u0, source=(0.0, 0.0, 0.0), t=0):
    """Pull streaming f_i(x) = fhat_i(x - c_i) with the boundary rule (t: the
    time of the post-collision state)."""
    f = post
    out = np.empty_like(f)
    if bc == "periodic":
        for i in range(9):
            out[i] = np.roll(post[i], shift=(C[i, 1], C[i, 0]), axis=(0, 1))
    elif bc == "channel":
        _, ny, nx = f.shape
        fs = feq(source_rho(source, rho0, t), *u0)
        for i in range(9):
            cx, cy = C[i]
            for iy in range(ny):
                sy = (iy - cy) % ny
                for ix in range(nx):
                    sx = ix - cx
                    if sx < 0:
                        out[i, iy, ix] = fs[i]
                    elif sx >= nx:
                        out[i, iy, ix] = post[i, sy, nx - 1]
                    else:
                        out[i, iy, ix] = post[i, sy, sx]
    else:
        _, ny, nx = f.shape
        fb = feq(rho0, *u0)
        for i in range(9):
            cx, cy = C[i]
            for iy in range(ny):
                for ix in range(nx):
                    sx, sy = ix - cx, iy - cy
                    out[i, iy, ix] = post[i, sy, sx] if (0 <= sx < nx and 0 <= sy < ny) else fb[i]
    return out
