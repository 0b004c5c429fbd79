"""Von Neumann analysis of the linearised scheme (Sec. 3.2).

TEST INFRASTRUCTURE (see the package docstring).  Written from the analytic
derivatives of the collision, not from the oracle's step code, so that the
oracle's plane-wave response can be checked against it.

Linearising Eq. (app:Common) about a uniform state f^f = f^eq(rho^f, u^f)
(Eq. eq:linearized) gives delta f(x + c_i, t + 1)_i = (J delta f(x, t))_i with

    J = I + Lambda (E - I) + T,

    E_ij = d f^eq_i(rho*, j*) / d f_j
         = A_i / (1 + n chi) + (B_i . c_j) / (1 + m chi),
    A_i  = w_i (1 - 9/2 (c_i.u)^2 + 3/2 u.u),
    B_i  = w_i (3 c_i + 9 (c_i.u) c_i - 3 u),

where the 1/(1 + n chi), 1/(1 + m chi) factors are d rho*/d rho and
d j*/d j of the Guo parameterisation solved for rho*, j*.  The damping term
contributes T = -chi I (type I, f* = f), T = -chi E (type II) or
T = -chi L with L_ij = w_i (1/(1 + n chi) + 3 c_i.c_j / (1 + m chi))
(type III, linear equilibria).  Lambda = M^{-1} S M (App. A.1).

A plane wave delta f = A exp(i(k.x - w t)) (Eq. perturb-w-f) satisfies the
eigenproblem exp(-i w) A = G(k) A with G(k) = diag(exp(-i k.c_i)) J
(Eq. sec:matrix); lambda = exp(-i w) is the amplification factor per step.
"""
from __future__ import annotations

import numpy as np

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
C = np.stack([M[1], M[2]], axis=1)  # [9, 2]
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def rates(s: float, s_c: float | None = None) -> np.ndarray:
    """Nine rates: s_c on the conserved rows 0..2 (default s_c = s), s elsewhere."""
    sc = s if s_c is None else s_c
    return np.array([sc, sc, sc, s, s, s, s, s, s], dtype=np.float64)


def jacobian(variant: str, s9, chi: float, n: float = 0.5, m: float = 0.5,
             rho_f: float = 1.0, u_f=(0.0, 0.0)) -> np.ndarray:
    """J = d(post-collision f)/d f at f = f^eq(rho^f, u^f), 9x9."""
    u = np.asarray(u_f, dtype=np.float64)
    cu = C @ u
    A = W * (1 - 4.5 * cu**2 + 1.5 * (u @ u))
    B = W[:, None] * (3 * C + 9 * cu[:, None] * C - 3 * u[None, :])
    E = A[:, None] / (1 + n * chi) + (B @ C.T) / (1 + m * chi)
    lam = np.linalg.inv(M) @ np.diag(np.asarray(s9, dtype=np.float64)) @ M
    eye = np.eye(9)
    if variant == "I":
        T = -chi * eye
    elif variant == "II":
        T = -chi * E
    elif variant == "III":
        L = W[:, None] * (1 / (1 + n * chi) + 3 * (C @ C.T) / (1 + m * chi))
        T = -chi * L
    elif variant == "none":
        T = np.zeros((9, 9))
    else:
        raise ValueError(variant)
    return eye + lam @ (E - eye) + T


def amplification(k, J: np.ndarray) -> np.ndarray:
    """G(k) = diag(exp(-i k.c_i)) J for a wave vector k = (k_x, k_y)."""
    phase = np.exp(-1j * (C @ np.asarray(k, dtype=np.float64)))
    return phase[:, None] * J


def spectrum(k, J: np.ndarray) -> np.ndarray:
    return np.linalg.eigvals(amplification(k, J))


def max_growth(variant: str, s: float, chi: float, u_f=(0.0, 0.0), theta: float = 0.0,
               nk: int = 400, n: float = 0.5, m: float = 0.5, s_c: float | None = None) -> float:
    """max over |k| in (0, pi] along direction theta (Eq. wavenumber) of max_i |lambda_i(k)|."""
    J = jacobian(variant, rates(s, s_c), chi, n, m, 1.0, u_f)
    best = 0.0
    for kk in np.linspace(np.pi / nk, np.pi, nk):
        k = (kk * np.cos(theta), kk * np.sin(theta))
        best = max(best, float(np.max(np.abs(spectrum(k, J)))))
    return best


# ---------------------------------------------------------------------------
# Stability maps (the critical damping strength of Sec. 3.3 as a function of
# the rates, the target flow and the wave direction).
#
# growth(): the largest |lambda| over the wave numbers
#     k_j = (pi j / nk) (cos theta, sin theta),  j = 0 .. nk,
# i.e. the uniform mode (which carries the chi <= 4/s limit of
# Eq. criticalchi) and nk wave numbers up to the grid's cut-off pi.
#
# chi_crit(): the smallest damping strength at which the scheme turns
# unstable, found the plain way.  chi is scanned on nscan equally spaced
# values of [chi_lo, chi_hi]; "unstable" means growth > 1 + tol.  If the
# first value is already unstable the result is -inf; if no value is, +inf.
# Otherwise the interval between the last stable and the first unstable scan
# value is halved `iters` times and its midpoint returned.
# ---------------------------------------------------------------------------

def wavenumbers(nk: int, theta: float) -> np.ndarray:
    """[nk + 1, 2]: k_j = (pi j / nk)(cos theta, sin theta), j = 0..nk (k = 0 only
    when nk = 0)."""
    mag = np.array([0.0]) if nk == 0 else np.pi * np.arange(nk + 1) / nk
    return mag[:, None] * np.array([np.cos(theta), np.sin(theta)])[None, :]


def growth(variant: str, s9, chi: float, n: float = 0.5, m: float = 0.5, u_f=(0.0, 0.0),
           theta: float = 0.0, nk: int = 400, rho_f: float = 1.0):
    """(max_j max_i |lambda_i(G(k_j))|, |k_j| at which it occurs) over wavenumbers()."""
    J = jacobian(variant, s9, chi, n, m, rho_f, u_f)
    best, kbest = -1.0, 0.0
    for k in wavenumbers(nk, theta):
        g = float(np.max(np.abs(spectrum(k, J))))
        if g > best:
            best, kbest = g, float(np.hypot(*k))
    return best, kbest


def chi_crit(variant: str, s9, n: float = 0.5, m: float = 0.5, u_f=(0.0, 0.0),
             theta: float = 0.0, nk: int = 400, chi_lo: float = 0.0, chi_hi: float = 8.0,
             nscan: int = 17, iters: int = 40, tol: float = 1e-9) -> float:
    """Critical damping strength by scan and bisection (see the block comment)."""
    def unstable(chi):
        return growth(variant, s9, chi, n, m, u_f, theta, nk)[0] > 1.0 + tol

    grid = chi_lo + (chi_hi - chi_lo) * np.arange(nscan) / (nscan - 1)
    if unstable(grid[0]):
        return -np.inf
    for g in range(1, nscan):
        if unstable(grid[g]):
            a, b = grid[g - 1], grid[g]
            break
    else:
        return np.inf
    for _ in range(iters):
        mid = 0.5 * (a + b)
        if unstable(mid):
            b = mid
        else:
            a = mid
    return 0.5 * (a + b)
