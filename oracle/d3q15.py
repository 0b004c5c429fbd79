"""Oracle of the three-dimensional scheme: D3Q15 MRT with the absorbing-layer
damping terms, in plain FP64 NumPy.

TEST INFRASTRUCTURE (see the package docstring): only tests/, the smoke check
and bench.py's CPU legs use it.  It shares nothing with the CUDA path.

The definition is that of the two-dimensional oracle, Eq. (blbs-abc-1) with
Gamma = chi I, carried to fifteen velocities:

    f_i(x + c_i, t + 1) = f_i + Lambda_ij (f^eq_j(rho*, u*) - f_j) + T_i,
    Lambda = M^-1 S M   (M of App. A.2),
    rho* = (rho + n chi rho^f) / (1 + n chi),  j* = (j + m chi rho^f u^f) / (1 + m chi),
    T = chi (f^eq(q^f) - f)                   type I   (Sec. 2.2.1)
        chi (f^eq(q^f) - f^eq(rho*, u*))      type II  (Sec. 2.2.2)
        chi (f^Leq(q^f) - f^Leq(rho*, j*))    type III (Sec. 2.2.3)
        0                                     none,

worked in population space with Lambda formed explicitly.  The velocity set is
read off rows 1-3 of M.  The paper prints no D3Q15 weights or equilibrium:
this file takes the standard ones, w = 2/9 (rest), 1/9 (axes), 1/72
(diagonals), which give c_s^2 = 1/3 and fourth-order isotropy (pinned), and
the same second-order equilibrium and linear equilibrium as in 2-D.

Boundaries as in 2-D: "dirichlet" gives every population streaming in from
outside the lattice the value f^eq(rho0, u0), at every time level including
t = 0; "periodic" wraps all three axes.

Layout: f[i, z, y, x] (x fastest), i in the column order of M.
"""
from __future__ import annotations

import numpy as np

# App. A.2: the D3Q15 transformation matrix, row by row.
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
        [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1],
        [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1],
        [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1],
        [-2, -1, -1, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1],
        [16, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1],
        [0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1],
        [0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1],
        [0, 0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1],
        [0, 2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1],
    ],
    dtype=np.float64,
)
Q = 15
C = M[1:4].T.astype(int)  # [15, 3]: c_i = (M[1,i], M[2,i], M[3,i])
W = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
VARIANTS = ("none", "I", "II", "III")


def rates(s: float, s_c: float | None = None) -> np.ndarray:
    """Fifteen rates: s_c on the conserved rows 0..3 (default s), s elsewhere."""
    sc = s if s_c is None else s_c
    return np.array([sc] * 4 + [s] * 11, dtype=np.float64)


def _shape(a, nd):
    return a.reshape((Q,) + (1,) * nd)


def feq(rho, u):
    """f^eq_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u); rho[...], u[3, ...]."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    nd = rho.ndim
    cu = sum(_shape(C[:, a].astype(np.float64), nd) * u[a] for a in range(3))
    uu = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    return _shape(W, nd) * rho * (1 + 3 * cu + 4.5 * cu**2 - 1.5 * uu)


def feq_linear(rho, j):
    """f^Leq_i = w_i (rho + 3 c.j)."""
    rho = np.asarray(rho, dtype=np.float64)
    j = np.asarray(j, dtype=np.float64)
    nd = rho.ndim
    cj = sum(_shape(C[:, a].astype(np.float64), nd) * j[a] for a in range(3))
    return _shape(W, nd) * (rho + 3 * cj)


def lambda_matrix(s) -> np.ndarray:
    return np.linalg.inv(M) @ np.diag(np.asarray(s, dtype=np.float64)) @ M


class Problem:
    """A D3Q15 lattice problem: sizes, the fifteen rates in the row order of M
    (s[0:4] on the conserved rows), Guo weights n, m, variant, boundary, far
    field (rho0, u0), reference state (rho_f, u_f) and per-axis absorbing
    strengths (chi = max of the three at a cell)."""

    def __init__(self, nx, ny, nz, s, n=0.5, m=0.5, variant="II", bc="dirichlet", rho0=1.0,
                 u0=(0.0, 0.0, 0.0), rho_f=None, u_f=None, chi_x=None, chi_y=None, chi_z=None):
        if variant not in VARIANTS:
            raise ValueError(variant)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.s = np.broadcast_to(np.asarray(s, dtype=np.float64), (Q,)).copy()
        self.n, self.m = float(n), float(m)
        self.variant, self.bc = variant, bc
        self.rho0, self.u0 = float(rho0), np.asarray(u0, dtype=np.float64)
        self.rho_f = self.rho0 if rho_f is None else float(rho_f)
        self.u_f = self.u0 if u_f is None else np.asarray(u_f, dtype=np.float64)
        self.chi_x = np.zeros(nx) if chi_x is None else np.asarray(chi_x, dtype=np.float64)
        self.chi_y = np.zeros(ny) if chi_y is None else np.asarray(chi_y, dtype=np.float64)
        self.chi_z = np.zeros(nz) if chi_z is None else np.asarray(chi_z, dtype=np.float64)
        self.lam = lambda_matrix(self.s)

    def chi(self) -> np.ndarray:
        """chi[z, y, x] = max(chi_x[x], chi_y[y], chi_z[z]); zero everywhere when
        no damping term is selected (Gamma = 0 gives F = 0 in Eq. blbs, so also
        rho* = rho, j* = j)."""
        if self.variant == "none":
            return np.zeros((self.nz, self.ny, self.nx))
        return np.maximum(np.maximum(self.chi_x[None, None, :], self.chi_y[None, :, None]),
                          self.chi_z[:, None, None])

    def boundary_value(self) -> np.ndarray:
        return feq(np.float64(self.rho0), self.u0)


def _inflow_masks(shape):
    """For each i, the [z, y, x] mask of cells whose upstream cell x - c_i lies
    outside the lattice."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for i in range(Q):
        sx, sy, sz = x - C[i, 0], y - C[i, 1], z - C[i, 2]
        out.append((sx < 0) | (sx >= nx) | (sy < 0) | (sy >= ny) | (sz < 0) | (sz >= nz))
    return out


def stream(post: np.ndarray, prob: Problem) -> np.ndarray:
    """f_i(x) = post_i(x - c_i); outside the lattice: the boundary rule."""
    f = np.empty_like(post)
    for i in range(Q):
        f[i] = np.roll(post[i], shift=(C[i, 2], C[i, 1], C[i, 0]), axis=(0, 1, 2))
    if prob.bc == "dirichlet":
        fb = prob.boundary_value()
        for i, mask in enumerate(_inflow_masks(post.shape[1:])):
            f[i][mask] = fb[i]
    elif prob.bc != "periodic":
        raise ValueError(prob.bc)
    return f


def collide(f: np.ndarray, prob: Problem) -> np.ndarray:
    """Post-collision populations of every cell (no streaming)."""
    chi = prob.chi()
    rho = f.sum(axis=0)
    j = np.stack([np.tensordot(C[:, a].astype(np.float64), f, axes=(0, 0)) for a in range(3)])
    rs = (rho + prob.n * chi * prob.rho_f) / (1 + prob.n * chi)
    js = (j + prob.m * chi * prob.rho_f * prob.u_f[:, None, None, None]) / (1 + prob.m * chi)
    us = js / rs
    fe = feq(rs, us)
    post = f + np.tensordot(prob.lam, fe - f, axes=(1, 0))
    if prob.variant == "I":
        post += chi * (feq(np.float64(prob.rho_f), prob.u_f)[:, None, None, None] - f)
    elif prob.variant == "II":
        post += chi * (feq(np.float64(prob.rho_f), prob.u_f)[:, None, None, None] - fe)
    elif prob.variant == "III":
        jf = prob.rho_f * prob.u_f
        post += chi * (feq_linear(np.float64(prob.rho_f), jf)[:, None, None, None]
                       - feq_linear(rs, js))
    return post


class State:
    """Populations f[15, nz, ny, nx] (FP64, full values) of one problem."""

    def __init__(self, prob: Problem, rho, u):
        """f = f^eq(rho, u) at every cell (rho[nz, ny, nx], u[3, nz, ny, nx] or
        broadcastable), then the boundary rule for populations entering from
        outside."""
        self.prob = prob
        shp = (prob.nz, prob.ny, prob.nx)
        rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), shp)
        u = np.stack([np.broadcast_to(np.asarray(u[a], dtype=np.float64), shp) for a in range(3)])
        self.f = feq(rho, u)
        if prob.bc == "dirichlet":
            fb = prob.boundary_value()
            for i, mask in enumerate(_inflow_masks(shp)):
                self.f[i][mask] = fb[i]
        self.t = 0

    def run(self, nsteps: int) -> "State":
        for _ in range(nsteps):
            self.f = stream(collide(self.f, self.prob), self.prob)
            self.t += 1
        return self

    def moments(self):
        """(rho - rho0, u_x, u_y, u_z), each [nz, ny, nx]."""
        rho = self.f.sum(axis=0)
        u = [np.tensordot(C[:, a].astype(np.float64), self.f, axes=(0, 0)) / rho
             for a in range(3)]
        return (rho - self.prob.rho0, *u)


def gaussian_pulse(nx, ny, nz, x0, y0, z0, eps, b):
    """rho' = eps exp(-ln2 r^2 / b^2) around (x0, y0, z0) (b the half width at half
    maximum, as in the 2-D pulse of Sec. 4.1), [nz, ny, nx]."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - x0) ** 2 + (y - y0) ** 2 + (z - z0) ** 2
    return eps * np.exp(-np.log(2.0) * r2 / b**2)


def spherical_pulse(r, t, eps, b, cs=1.0 / np.sqrt(3.0)):
    """Inviscid linear acoustics in 3-D from a Gaussian rho'(r, 0) = g(r) at rest:
    r rho' satisfies the 1-D wave equation, so
    rho'(r, t) = [(r - ct) g(r - ct) + (r + ct) g(r + ct)] / (2 r),
    with g extended evenly (its value at r = 0 by the limit r -> 0)."""
    r = np.asarray(r, dtype=np.float64)
    a = np.log(2.0) / b**2

    def g(x):
        return eps * np.exp(-a * x * x)

    ct = cs * t
    with np.errstate(invalid="ignore", divide="ignore"):
        out = ((r - ct) * g(r - ct) + (r + ct) * g(r + ct)) / (2 * r)
    # r -> 0: d/dr [r g(r - ct)] style limit: g(ct) + ct g'(ct) ... = g(ct)(1 - 2 a (ct)^2)
    lim = g(ct) * (1 - 2 * a * ct * ct)
    return np.where(r == 0, lim, out)
