"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle (or the Von Neumann tool / pulse solution it is
checked with) to something other than itself: a value or statement printed in
the paper (tests/golden/), a closed form, an invariant, or brute force.  The
plausible mistakes each one catches are named in its docstring.
"""
import math

import numpy as np
import pytest

from conftest import golden_rows

import workloads as wl


def _prob(core, nx, ny, s, **kw):
    return core.Problem(nx, ny, np.asarray(s, dtype=np.float64), **kw)


# ---------------------------------------------------------------- algebra ----

def test_transformation_matrix_is_the_papers(oracle_lib):
    """The oracle's M equals App. A.1 and its velocity set is rows 1-2 of it.
    Catches a mistyped entry or a permuted velocity order."""
    cx, cy, w, mm = oracle_lib.tables()
    golden = np.array([[float(v) for v in r] for r in golden_rows("d2q9_transformation_matrix.txt")])
    assert golden.shape == (9, 9)
    np.testing.assert_array_equal(mm, golden)
    np.testing.assert_array_equal(cx, golden[1])
    np.testing.assert_array_equal(cy, golden[2])
    # rows are mutually orthogonal: M M^T = diag(9, 6, 6, 36, 36, 12, 12, 4, 4)
    np.testing.assert_array_equal(golden @ golden.T, np.diag([9, 6, 6, 36, 36, 12, 12, 4, 4]))


def test_weights_reproduce_the_papers_sound_speed(oracle_lib):
    """Sec. 4.2 prints lambda = c_s / 2 = 0.288675; the D2Q9 weights must give that
    c_s (second moment) and be isotropic to fourth order.  Catches wrong weights."""
    cx, cy, w, _ = oracle_lib.tables()
    rows = dict((r[0], float(r[1])) for r in golden_rows("line_source_wavelength.txt"))
    cs = 2 * rows["lambda"]
    c = np.stack([cx, cy], 1).astype(float)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    np.testing.assert_allclose(second, cs**2 * np.eye(2), rtol=2e-6)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(fourth, iso, atol=1e-15)
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16


def test_equilibrium_moments_closed_form(oracle_lib):
    """f^eq has the Navier-Stokes moments rho, rho u, rho c_s^2 I + rho u u; its linear
    part has rho, j, rho c_s^2 I with no rho u u term (the point of the type III term,
    Sec. 2.2.3).  Catches a wrong coefficient or sign in either equilibrium."""
    cx, cy, _, _ = oracle_lib.tables()
    c = np.stack([cx, cy], 1).astype(float)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.2, 0.2, 2)
        fe = oracle_lib.feq(rho, *u)
        assert fe.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(c.T @ fe, rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", fe, c, c)
        np.testing.assert_allclose(pi, rho / 3 * np.eye(2) + rho * np.outer(u, u), atol=1e-15)
        j = rho * u
        fl = oracle_lib.feq_linear(rho, *j)
        assert fl.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(c.T @ fl, j, atol=1e-15)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", fl, c, c), rho / 3 * np.eye(2), atol=1e-15)


def test_lambda_is_bgk_when_rates_are_equal(oracle_lib):
    """Lambda = M^{-1} S M reduces to s I (Eq. eq_BGK_LBM_R) when all rates are equal,
    and has the rows of M as left eigenvectors with eigenvalues s_k otherwise."""
    lam = oracle_lib.lambda_matrix(np.full(9, 1.7))
    np.testing.assert_allclose(lam, 1.7 * np.eye(9), atol=1e-14)
    s = np.array([1.1, 1.2, 1.3, 1.4, 1.5, 1.6, 1.7, 1.8, 1.9])
    lam = oracle_lib.lambda_matrix(s)
    _, _, _, mm = oracle_lib.tables()
    np.testing.assert_allclose(mm @ lam, np.diag(s) @ mm, atol=1e-13)


# ----------------------------------------------------- invariants / k = 0 ----

@pytest.mark.parametrize("rates", ["bgk", "mrt"])
def test_mass_and_momentum_conserved_without_damping(oracle_lib, rates):
    """chi = 0 and periodic walls: sum rho and sum j are invariants of the scheme
    (Eq. eq_conservative).  Catches a streaming or collision error that leaks mass."""
    s = np.full(9, 1.9) if rates == "bgk" else np.array([1.9, 1.9, 1.9, 1.2, 1.5, 1.7, 1.7, 1.9, 1.9])
    prob = _prob(oracle_lib, 24, 17, s, variant="II", bc="periodic", u0=(0.05, -0.02),
                 u_f=(0.05, -0.02))
    rng = np.random.default_rng(2)
    rho = 1 + 1e-3 * rng.standard_normal((17, 24))
    st = oracle_lib.State(prob, rho, 0.05 + 1e-3 * rng.standard_normal((17, 24)),
                          -0.02 + 1e-3 * rng.standard_normal((17, 24)))
    f0 = st.f.copy()
    cx, cy, _, _ = oracle_lib.tables()
    st.run(300)
    for a, b in ((f0.sum(), st.f.sum()),
                 (np.tensordot(cx, f0, 1).sum(), np.tensordot(cx, st.f, 1).sum()),
                 (np.tensordot(cy, f0, 1).sum(), np.tensordot(cy, st.f, 1).sum())):
        assert abs(a - b) <= 1e-13 * f0.sum()


def _uniform_state(core, prob, drho=0.0, dmom=None):
    f = np.broadcast_to(core.feq(prob.rho_f, *prob.u_f)[:, None, None],
                        (9, prob.ny, prob.nx)).copy()
    cx, cy, w, mm = core.tables()
    minv = np.linalg.inv(mm)
    dm = np.zeros(9)
    dm[0] = drho
    if dmom is not None:
        k, amp = dmom
        dm[k] = amp
    f += (minv @ dm)[:, None, None]
    st = core.State(prob, np.ones((prob.ny, prob.nx)), 0.0, 0.0)
    st.f[:] = f
    return st, mm


@pytest.mark.parametrize("variant", ["I", "II", "III"])
@pytest.mark.parametrize("chi", [0.3, 1.2, 4 / 1.9 - 0.05, 4 / 1.9 + 0.05])
def test_uniform_density_decay_closed_form(oracle_lib, variant, chi):
    """k = 0 mode (a uniform density excess on a periodic lattice).  Solving the Guo
    definitions for rho* and relaxing the conserved row with s_c gives per step
        types II, III: lambda = (1 + n chi - s_c n chi - chi) / (1 + n chi)
        type I:        lambda = 1 - s_c n chi / (1 + n chi) - chi
    and for n = 1/2, s_c = s the II/III factor leaves [-1, 1] exactly when
    chi > 4/s (Eq. criticalchi).  Catches a wrong rho* (explicit instead of
    implicit), a dropped n, or a sign error in the damping term."""
    s, n = 1.9, 0.5
    prob = _prob(oracle_lib, 3, 2, np.full(9, s), variant=variant, bc="periodic",
                 chi_x=np.full(3, chi), chi_y=np.full(2, chi), n=n, m=n)
    st, mm = _uniform_state(oracle_lib, prob, drho=1e-2)
    if variant == "I":
        lam = 1 - s * n * chi / (1 + n * chi) - chi
    else:
        lam = (1 + n * chi - s * n * chi - chi) / (1 + n * chi)
    steps = 6
    st.run(steps)
    drho = st.f.sum(0) - 1.0
    np.testing.assert_allclose(drho, 1e-2 * lam**steps, rtol=1e-9, atol=1e-15)
    if variant != "I":
        assert (abs(lam) <= 1.0) == (chi <= 4 / s)


@pytest.mark.parametrize("variant", ["none", "I", "II", "III", "viscous"])
def test_non_conserved_moment_decay(oracle_lib, variant):
    """A uniform excess in a non-conserved moment m_k relaxes by (1 - s_k) per step,
    by (1 - s_k - chi) with the type I term (s' = s + chi, Eq. effectrelax), and by
    (1 - s_k') with the viscosity sponge of Sec. 4.1 at layer fraction r,
    s_k' = s_k + (1 - s_k) r.  Catches a Lambda built with the wrong row order, a
    type I term that does not act on f itself, or a sponge ramp that also moves the
    conserved rows."""
    s = np.array([1.8, 1.8, 1.8, 1.1, 1.3, 1.5, 1.5, 1.7, 1.7])
    chi = 0.0 if variant == "none" else 0.2
    prob = _prob(oracle_lib, 2, 2, s, variant=variant if variant != "none" else "none",
                 bc="periodic", chi_x=np.full(2, chi), chi_y=np.full(2, chi))
    for k in range(3, 9):
        st, mm = _uniform_state(oracle_lib, prob, dmom=(k, 1e-2))
        base = mm @ oracle_lib.feq(1.0, 0.0, 0.0)
        st.run(3)
        m_now = mm @ st.f[:, 0, 0] - base
        fac = 1 - s[k] - (chi if variant == "I" else 0.0)
        if variant == "viscous":
            fac = 1 - (s[k] + (1 - s[k]) * chi)
        expect = np.zeros(9)
        expect[k] = 1e-2 * fac**3
        np.testing.assert_allclose(m_now, expect, rtol=1e-12, atol=5e-15)


# ---------------------------------------------------------- Von Neumann ----

def _chi_expr(expr, s):
    return float(eval(expr, {"__builtins__": {}}, {"s": s}))


def test_von_neumann_reproduces_the_papers_stability_claims():
    """Every stability statement of Sec. 3.3 (Figs. 1-4, 8, 9) holds for the
    linearised scheme.  Pins the readings rho* implicit and s_c = s: the explicit
    rho* or s_c = 0 move or remove the chi = 4/s threshold."""
    from oracle import vonneumann as vn

    rows = golden_rows("stability_claims.txt")
    assert len(rows) == 12
    for r in rows:
        variant, s = r[0], float(r[1])
        chi = _chi_expr(r[2], s)
        g = vn.max_growth(variant, s, chi, (float(r[3]), float(r[4])), theta=0.0, nk=300)
        verdict = r[5]
        if verdict == "stable":
            assert g < 1 - 1e-6, (r, g)
        elif verdict == "marginal":
            assert abs(g - 1) < 1e-9, (r, g)
        else:
            assert g > 1 + 1e-6, (r, g)


def test_von_neumann_small_k_matches_navier_stokes_modes():
    """chi = 0, small k: the eigenvalues lambda = exp(-i omega) give the acoustic and
    shear modes of Eq. (th:d): Re omega = +-c_s|k| + u.k, u.k and Im omega = -nu k^2
    for both (D2Q9 BGK: bulk viscosity = shear viscosity in 2-D), nu = (1/s - 1/2)/3."""
    from oracle import vonneumann as vn

    s, u = 1.8, np.array([0.05, 0.0])
    nu = (1 / s - 0.5) / 3
    J = vn.jacobian("none", vn.rates(s), 0.0, u_f=tuple(u))
    for kk in (0.01, 0.02):
        k = np.array([kk, 0.0])
        lam = vn.spectrum(k, J)
        lam = lam[np.argsort(-np.abs(lam))][:3]  # hydrodynamic modes
        omega = 1j * np.log(lam)
        re = np.sort(omega.real)
        cs = 1 / math.sqrt(3)
        np.testing.assert_allclose(re, np.sort([-cs * kk + u @ k, u @ k, cs * kk + u @ k]),
                                   atol=5 * kk**3 + 2e-3 * kk**2)
        np.testing.assert_allclose(omega.imag, -nu * kk**2, rtol=0.05)


def test_critical_chi_map_closed_forms():
    """The stability map's critical chi (scan over [0, 8] then bisection, growth
    over k_j = pi j / nk including the uniform mode) against what Sec. 3.3 fixes:
    type II with equal rates turns unstable at 4/s (Eq. criticalchi), type I at
    2 - s (Eq. effectrelax, Fig. 1a), type II keeps 4/s with u^f = (0.1, 0)
    (Fig. 8), type III with u^f = (0.1, 0) lies between 2.5/s and 3/s (Fig. 9).
    For type II both the uniform mode and the k = pi mode along x turn critical
    at 4/s, so the coarse grid nk = 4 finds it as well as nk = 64."""
    from oracle import vonneumann as vn

    for s in (1.5, 1.9, 1.99):
        for nk in (4, 64):
            c = vn.chi_crit("II", vn.rates(s), nk=nk, iters=34)
            assert abs(c - 4 / s) < 1e-6, (s, nk, c)
        c = vn.chi_crit("I", vn.rates(s), nk=64, chi_hi=1.0, iters=34)
        assert abs(c - (2 - s)) < 1e-6, (s, c)
    c = vn.chi_crit("II", vn.rates(1.99), u_f=(0.1, 0.0), nk=64, iters=34)
    assert abs(c - 4 / 1.99) < 1e-6, c
    c = vn.chi_crit("III", vn.rates(1.99), u_f=(0.1, 0.0), nk=64, chi_hi=4.0, iters=34)
    assert 2.5 / 1.99 < c < 3 / 1.99, c
    # the s_c = 0 reading moves the threshold far above 4/s (reading C3)
    assert vn.chi_crit("II", vn.rates(1.99, 0.0), nk=64, iters=20) > 4 / 1.99 + 0.1
    # end cases of the scan
    assert vn.chi_crit("I", vn.rates(1.99), nk=8, chi_lo=0.05, chi_hi=1.0) == -np.inf
    assert vn.chi_crit("II", vn.rates(1.9), nk=8, chi_hi=2.0) == np.inf


def test_growth_on_the_wavenumber_grid():
    """k_j runs over pi j / nk along theta and includes k = 0: with chi = 0 the
    conserved modes give growth exactly 1 (Eq. th:d at k = 0); for the uniform
    mode alone (nk = 0) type II gives the closed form of Eq. criticalchi,
    |1 + n chi - s n chi - chi| / (1 + n chi), reached at k = 0."""
    from oracle import vonneumann as vn

    k = vn.wavenumbers(4, np.pi / 6)
    np.testing.assert_allclose(np.hypot(k[:, 0], k[:, 1]), np.pi * np.arange(5) / 4, atol=1e-15)
    np.testing.assert_allclose(k[2], (np.pi / 2) * np.array([np.cos(np.pi / 6), np.sin(np.pi / 6)]))
    for s in (1.2, 1.9):
        g, _ = vn.growth("none", vn.rates(s), 0.0, u_f=(0.1, 0.05), theta=0.3, nk=32)
        assert abs(g - 1) < 1e-12, g
        for chi in (0.5, 4 / s + 0.2):
            # k = 0: the conserved modes decay by lam, the others by 1 - s
            g, kk = vn.growth("II", vn.rates(s), chi, nk=0)
            lam = (1 + 0.5 * chi - s * 0.5 * chi - chi) / (1 + 0.5 * chi)
            assert kk == 0.0 and abs(g - max(abs(lam), abs(1 - s))) < 1e-12, (s, chi, g, lam)


def test_critical_chi_bounds_with_distinct_rates():
    """Distinct MRT rates (App. A.1 S with s_e, s_eps, s_q, s_nu apart): the uniform
    mode alone fixes upper bounds on the critical chi, so the map can never lie
    above them: type II at most 4/s_c (Eq. criticalchi with the conserved rate),
    type I at most 2 - max s_k over the non-conserved rates (Eq. effectrelax).
    Checked on seeded random rates, target flows and directions."""
    from oracle import vonneumann as vn

    rng = np.random.default_rng(11)
    for _ in range(6):
        sc = rng.uniform(1.2, 1.99)
        s9 = np.concatenate([[sc] * 3, rng.uniform(1.0, 1.99, 6)])
        uf = tuple(rng.uniform(-0.1, 0.1, 2))
        th = rng.uniform(0, np.pi / 2)
        c2 = vn.chi_crit("II", s9, u_f=uf, theta=th, nk=32, iters=24)
        assert c2 <= 4 / sc + 1e-6, (s9, c2)
        c1 = vn.chi_crit("I", s9, u_f=uf, theta=th, nk=32, chi_hi=1.0, iters=24)
        assert c1 <= 2 - s9[3:].max() + 1e-6, (s9, c1)


@pytest.mark.parametrize("variant,s,chi,uf", [
    ("II", 1.99, 4 / 1.99 - 0.1, (0.0, 0.0)),
    ("I", 1.9, 0.1, (0.0, 0.0)),
    ("III", 1.99, 3 / 1.99, (0.1, 0.0)),
    ("none", 1.988, 0.0, (0.05, 0.0)),
    ("II", 1.5, 0.7, (0.1, 0.0)),
])
def test_plane_wave_follows_von_neumann(oracle_lib, variant, s, chi, uf):
    """Seed each eigenvector of G(k), k = (2 pi / N, 0), on a periodic lattice with
    uniform chi and run N steps of the oracle: the linear response (difference of
    +-eps runs) must be lambda^N times the seed.  Ties the oracle's full step
    (moments, rho*, collision, damping, streaming direction) to the analytic
    linearisation of Sec. 3.2."""
    from oracle import vonneumann as vn

    N, eps = 32, 1e-5
    J = vn.jacobian(variant, vn.rates(s), chi, 0.5, 0.5, 1.0, uf)
    k = 2 * np.pi / N
    lam, V = np.linalg.eig(vn.amplification((k, 0.0), J))
    x = np.arange(N)
    base = oracle_lib.feq(1.0, *uf)
    prob = _prob(oracle_lib, N, 1, vn.rates(s), variant=variant, bc="periodic", u0=uf, u_f=uf,
                 chi_x=np.full(N, chi), chi_y=np.full(1, chi))
    for idx in range(9):
        A = V[:, idx]
        seed = np.real(A[:, None] * np.exp(1j * k * x)[None, :])
        outs = []
        for sg in (1, -1):
            st = oracle_lib.State(prob, np.ones((1, N)), uf[0], uf[1])
            st.f[:] = base[:, None, None] + sg * eps * seed[:, None, :]
            st.run(N)
            outs.append(st.f[:, 0, :].copy())
        lin = (outs[0] - outs[1]) / (2 * eps)
        pred = np.real(lam[idx] ** N * A[:, None] * np.exp(1j * k * x)[None, :])
        assert np.abs(lin - pred).max() <= 1e-8 * np.abs(seed).max(), (idx, lam[idx])


# ------------------------------------------------------- acoustic pulse ----

def test_pulse_solution_at_t0_is_the_gaussian():
    """The Bessel integral of Sec. 4.1 at t = 0 is the Hankel transform pair of the
    initial Gaussian: rho'(r, 0) = eps exp(-alpha r^2)."""
    from oracle import pulse

    r = np.linspace(0, 20, 81)
    for b in (3.0, 5.0):
        got = pulse.rho_prime(r, 0 * r, 0.0, eps=1e-3, b=b)
        np.testing.assert_allclose(got, 1e-3 * np.exp(-math.log(2) / b**2 * r**2), atol=1e-15)


def _pulse_error(core, b, U0):
    from oracle import pulse

    eps, nu = 1e-6, 1e-5
    R = int(math.ceil(6 * b + 3.6 * b + 4))
    N = 2 * R + 1
    T = int(round(2 * b * math.sqrt(3)))
    prob = _prob(core, N, N, np.full(9, wl.rate_from_viscosity(nu)), variant="none",
                 u0=(U0, 0.0), u_f=(U0, 0.0))
    rho = 1 + wl.gaussian_pulse(N, N, R, R, eps, b)
    st = core.State(prob, rho, U0, 0.0).run(T)
    r, _, _ = st.moments()
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    return np.abs(r - pulse.rho_prime(X, Y, T, eps=eps, b=b, x0=R, y0=R, U0=U0)).max() / eps


@pytest.mark.parametrize("U0", [0.0, 0.05])
def test_pulse_converges_to_the_bessel_solution(oracle_lib, U0):
    """Interior of the 2-D acoustic pulse (Sec. 4.1) before any reflection, in the
    linear, nearly inviscid regime: the max error against the closed form falls at
    second order as the half-width b doubles (3 -> 6 -> 12 cells).  Catches a wrong
    sound speed, a wrong convection velocity, or a streaming direction error."""
    e = [_pulse_error(oracle_lib, b, U0) for b in (3.0, 6.0, 12.0)]
    assert e[0] < 0.02
    assert e[0] / e[1] > 3.5 and e[1] / e[2] > 3.5, e


# ------------------------------------------------------------ symmetry ----

def _run_workload(core, w, steps):
    prob = core.Problem(w.nx, w.ny, w.s, n=w.n, m=w.m, variant=w.variant, bc=w.bc, rho0=w.rho0,
                        u0=w.u0, rho_f=w.rho_f, u_f=w.u_f, chi_x=w.chi_x, chi_y=w.chi_y,
                        src_amp=w.source[0], src_omega=w.source[1], src_phase=w.source[2])
    return core.State(prob, *w.initial_fields()).run(steps)


@pytest.mark.parametrize("variant", ["none", "I", "II", "III"])
def test_mirror_symmetry(oracle_lib, variant):
    """u0 = 0, centred pulse, symmetric chi: rho' is invariant under the x-mirror,
    the y-mirror and the transpose (the D4 symmetry of the lattice and of the
    initial data).  With mean flow along x only the y-mirror survives.  Catches an
    asymmetric velocity table or an off-by-one in streaming or the layer."""
    w = wl.small_pulse(variant).with_(nx=60, ny=60, chi_x=wl.ramp_profile(60, 12, 0.1),
                                      chi_y=wl.ramp_profile(60, 12, 0.1))
    w.meta.update(x0=29.5, y0=29.5)
    # the oracle carries full populations (~rho0 = 1), so round-off is ~1e-16 absolute
    r, _, _ = _run_workload(oracle_lib, w, 60).moments()
    scale = np.abs(r).max()
    assert scale > 1e-5
    for img in (r[:, ::-1], r[::-1, :], r.T):
        assert np.abs(r - img).max() <= 1e-13
    w2 = w.with_(u0=(0.08, 0.0), u_f=(0.08, 0.0))
    r2, _, _ = _run_workload(oracle_lib, w2, 60).moments()
    assert np.abs(r2 - r2[::-1, :]).max() <= 1e-13
    assert np.abs(r2 - r2[:, ::-1]).max() > 1e-6 * np.abs(r2).max()


# ---------------------------------------------------------- brute force ----

@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 3), (1, 1), (2, 7)])
@pytest.mark.parametrize("variant", ["none", "I", "II", "III", "viscous"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "channel"])
def test_c_oracle_matches_numpy_twin(oracle_lib, nx, ny, variant, bc):
    """Tiny lattices, random populations, MRT rates, 3 steps: the C oracle equals the
    independent NumPy statement to round-off.  Catches indexing, layout and
    boundary mistakes in the C code.  The channel (line source, outflow,
    periodic y) runs its steps in two calls, which pins the source's clock."""
    from oracle import twin

    if bc == "channel" and nx < 2:
        pytest.skip("the channel's outflow needs two columns")
    rng = np.random.default_rng(nx * 100 + ny)
    s = np.array([1.6, 1.6, 1.6, 1.1, 1.2, 1.3, 1.3, 1.9, 1.9])
    u0 = (0.03, -0.01)
    src = (2e-3, 0.7, 0.3)
    chi_x = rng.uniform(0, 0.6, nx)
    chi_y = rng.uniform(0, 0.6, ny)
    prob = _prob(oracle_lib, nx, ny, s, variant=variant, bc=bc, n=0.4, m=0.6, rho0=1.0, u0=u0,
                 rho_f=1.01, u_f=(0.02, 0.01), chi_x=chi_x, chi_y=chi_y, src_amp=src[0],
                 src_omega=src[1], src_phase=src[2])
    rho = 1 + 0.01 * rng.standard_normal((ny, nx))
    ux = 0.03 + 0.01 * rng.standard_normal((ny, nx))
    uy = -0.01 + 0.01 * rng.standard_normal((ny, nx))
    st = oracle_lib.State(prob, rho, ux, uy)
    f = twin.init(rho, ux, uy, bc=bc, rho0=1.0, u0=u0, source=src)
    np.testing.assert_allclose(st.f, f, atol=1e-15)
    chi = np.maximum(chi_x[None, :], chi_y[:, None])
    for t in range(3):
        f = twin.step(f, chi, s, variant, n=0.4, m=0.6, rho_f=1.01, u_f=(0.02, 0.01), bc=bc,
                      rho0=1.0, u0=u0, source=src, t=t)
    st.run(2)
    st.run(1)
    np.testing.assert_allclose(st.f, f, atol=2e-15)


# ------------------------------------------------------------ line source ----

def _zero_crossings(y):
    """Positions (linear interpolation) where y crosses zero upwards."""
    i = np.nonzero((y[:-1] < 0) & (y[1:] >= 0))[0]
    return i + y[i] / (y[i] - y[i + 1])


@pytest.mark.parametrize("ux", [0.0, 0.1])
def test_line_source_emits_a_plane_wave_at_the_sound_speed(oracle_lib, ux):
    """Sec. 4.2: the line source rho0 + A sin(2 pi t / T) on the left edge of a
    y-periodic channel emits a plane wave.  The field does not depend on y, and
    behind the front the wavelength is (c_s + U) T, the downstream phase speed of
    linear acoustics in a mean flow U (c_s = 1/sqrt(3), Sec. 2.1).  Catches a
    source on the wrong populations, a wrong clock or a mis-wrapped y."""
    T = 100.0
    w = wl.line_source(nx=700, ny=3, variant="none", width=0, period=T, u0=(ux, 0.0), nu=2e-4)
    st = _run_workload(oracle_lib, w, 900)
    r = st.moments()[0]
    assert np.abs(r - r[0]).max() == 0.0
    x0 = _zero_crossings(r[0, 40:420])
    lam = np.diff(x0).mean()
    assert abs(lam - (wl.CS + ux) * T) < 0.01 * (wl.CS + ux) * T, (lam, (wl.CS + ux) * T)
    # the source drives an O(A) wave
    amp = np.abs(r[0, 40:420]).max()
    assert 0.3 * w.source[0] < amp < 1.5 * w.source[0]


def _line_source_error(core, variant, width, ux=0.0, nx=800):
    """Relative L2 error of rho' over the first 640 cells of the channel at the
    paper's sample time, against the same source in a channel long enough that
    nothing comes back from its far end before that time."""
    w = wl.line_source(nx=nx, ny=2, variant=variant, width=width, u0=(ux, 0.0))
    ref = wl.line_source(nx=1200, ny=2, variant="none", width=0, u0=(ux, 0.0), steps=w.steps)
    got = _run_workload(core, w, w.steps).moments()[0][0, :640]
    want = _run_workload(core, ref, w.steps).moments()[0][0, :640]
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


@pytest.mark.parametrize("ux", [0.0, 0.1])
def test_line_source_layer_removes_the_outflow_reflection(oracle_lib, ux):
    """Sec. 4.2 (Figs. 9-10): at t = T_o + 10 T_p the type II layer (chi = 4/s -
    0.001, 0.8 H = 160 cells) leaves the field in front of it almost exactly
    the unbounded solution, the outflow alone reflects strongly, the viscosity
    sponge lies in between, and a layer one wavelength thick (58 cells, about
    0.3 H) already does nearly as well as the full one."""
    e_none = _line_source_error(oracle_lib, "none", 0, ux)
    e_visc = _line_source_error(oracle_lib, "viscous", 160, ux)
    e_ii = _line_source_error(oracle_lib, "II", 160, ux)
    e_ii_thin = _line_source_error(oracle_lib, "II", 58, ux)
    # measured: none 0.22 / 0.15, viscous 0.14 / 0.10, type II 1.1e-4, one wavelength 5.3e-4
    assert e_ii < 0.002 * e_none, (e_ii, e_none)
    assert e_ii < e_visc < 0.8 * e_none, (e_ii, e_visc, e_none)
    assert e_ii_thin < 0.01 * e_none, (e_ii_thin, e_none)


# ------------------------------------------------------ absorption trends ----

def _reflected_energy(core, w, steps):
    from oracle import diagnostics as dg

    prob = core.Problem(w.nx, w.ny, w.s, variant=w.variant, bc=w.bc, u0=w.u0, u_f=w.u_f,
                        chi_x=w.chi_x, chi_y=w.chi_y)
    st = core.State(prob, *w.initial_fields())
    W = w.width
    reg = (W, W, w.nx - W, w.ny - W)
    e0 = dg.reduce_fields(*st.moments(), region=reg)[3]
    st.run(steps)
    r = st.moments()
    return dg.reduce_fields(*r, region=reg)[3] / e0, dg.e_l2(r[0])


def test_type_II_layer_suppresses_reflection(oracle_lib):
    """Figs. n3-n4: without a layer the pulse comes back from the Dirichlet walls;
    with the type II layer the interior energy left after the wave has passed is
    two orders of magnitude smaller."""
    w = wl.small_pulse("II", "f64")
    bare = w.with_(chi_x=np.zeros(100), chi_y=np.zeros(100), variant="none")
    r_bare, _ = _reflected_energy(oracle_lib, bare, 300)
    r_layer, _ = _reflected_energy(oracle_lib, w, 300)
    assert r_layer < 1e-2 * r_bare


def test_thicker_layer_absorbs_better(oracle_lib):
    """Fig. n7: E_L2 after the pulse has left falls as the layer thickens from 2b to
    3b to 4b (type II, Orszag profile of Eq. normalizedsigma, chi = 4/s - 0.001)."""
    out = []
    for W in (20, 30, 40):
        w = wl.pulse_workload(200, 200, variant="II", storage="f64", b=10.0, width=W, chi_max=0.0,
                              nu=1e-7)
        chi = 4 / w.s[0] - 0.001
        w = w.with_(chi_x=wl.orszag_profile(200, W, chi), chi_y=wl.orszag_profile(200, W, chi))
        out.append(_reflected_energy(oracle_lib, w, 600)[1])
    assert out[0] > out[1] > out[2], out


def _sweep_energies(core, w, steps=300, every=5, ring_steps=150):
    """(R, E_wall): the interior acoustic energy after `steps` over its initial value
    (reading C14), and the energy in the two cells next to the wall summed every
    `every` steps up to `ring_steps`, over the same initial value."""
    from helpers import interior_region, ring_regions, oracle_problem
    from oracle import diagnostics as dg

    st = core.State(oracle_problem(core, w), *w.initial_fields())
    reg = interior_region(w)
    e0 = dg.reduce_fields(*st.moments(), region=reg)[3]
    wall, t = 0.0, 0
    while t < ring_steps:
        st.run(every)
        t += every
        fields = st.moments()
        wall += every * sum(dg.reduce_fields(*fields, region=q)[3] for q in ring_regions(w.nx, w.ny))
    st.run(steps - t)
    return dg.reduce_fields(*st.moments(), region=reg)[3] / e0, wall / e0


def test_chi_sweep_toward_the_critical_strength(oracle_lib):
    """Type II on the 100 x 100 pulse, peak strength swept to 4/s - 0.001 (Sec. 4.1's
    choice; Eq. criticalchi).  What the paper's analysis fixes along the sweep:

    * every strength of the sweep removes the reflection: the interior energy left
      after 300 steps is more than 50x below no layer (Figs. n3-n4);
    * the energy that crosses the layer and reaches the wall falls by more than
      10^4 from chi_max = 0.1 to 0.5, then rises monotonically toward the critical
      strength.  The uniform mode's amplification per step in the layer,
      lambda_0 = (1 + n chi - s n chi - chi)/(1 + n chi) (Eq. criticalchi's
      closed form), vanishes at chi = 1/(n(s - 1) + 1) and reaches -1 at 4/s, the
      edge of stability: approaching it, the layer damps each step less.  The
      sweep's R therefore does not fall monotonically toward 4/s.

    Planted in a copy of the oracle, a lost type II term or one of the wrong sign
    fails it.  (The explicit reading of rho* passes here; the Von Neumann pins of
    the critical strength catch it.)"""
    sweep = wl.chi_sweep("f64")
    s = float(sweep[0].s[0])
    bare = sweep[0].with_(chi_x=np.zeros(100), chi_y=np.zeros(100), variant="none")
    r_none, wall_none = _sweep_energies(oracle_lib, bare)
    got = [_sweep_energies(oracle_lib, w) for w in sweep]
    R = np.array([g[0] for g in got])
    wall = np.array([g[1] for g in got])
    assert np.all(R < r_none / 50), (R, r_none)
    assert wall[0] < wall_none / 50 and wall[0] > 1e4 * wall[1], (wall, wall_none)
    assert np.all(np.diff(wall[1:]) > 0), wall
    lam0 = [(1 + 0.5 * c - s * 0.5 * c - c) / (1 + 0.5 * c) for c in (w.chi_max for w in sweep)]
    assert np.all(np.diff(np.abs(lam0[1:])) > 0) and abs(lam0[-1] + 1) < 1e-3, lam0


@pytest.mark.parametrize("rho0,uf", [(1.3, (0.0, 0.0)), (0.8, (0.08, 0.0))])
@pytest.mark.parametrize("direction", [1, -1])
def test_acoustic_energy_weights_by_equipartition(oracle_lib, rho0, uf, direction):
    """The acoustic energy of the diagnostics, c_s^2 rho'^2/(2 rho0) + rho0|u - u0|^2/2,
    pinned without restating it: a travelling sound wave carries equal potential and
    kinetic energy (rho' = rho0 |u'|/c_s), and a single mode of the linearised
    scheme (Sec. 3.2) loses energy exactly as |lambda|^2 per step.  The wave is the
    right- or left-running eigenvector of G(k), k = 2 pi/64, seeded on a periodic
    lattice (rho0 != 1, with and without mean flow).  Each term is taken alone by
    zeroing the other field.  A wrong c_s^2, a dropped 1/2, rho0 in the wrong place
    or |u| instead of |u - u0| breaks the balance by 20 % or more; the lattice's
    own dispersion leaves 2e-3."""
    from oracle import diagnostics as dg
    from oracle import vonneumann as vn

    N, eps, s = 64, 1e-6, 1.99
    k = 2 * np.pi / N
    J = vn.jacobian("none", vn.rates(s), 0.0, 0.5, 0.5, rho0, uf)
    lam, V = np.linalg.eig(vn.amplification((k, 0.0), J))
    want = -(uf[0] + direction / math.sqrt(3.0)) * k  # phase of exp(-i omega)
    idx = int(np.argmin(np.abs(np.angle(lam) - want) + 10 * np.abs(np.abs(lam) - 1)))
    seed = np.real(V[:, idx][:, None] * np.exp(1j * k * np.arange(N))[None, :])
    seed *= eps / np.abs(seed.sum(0)).max()
    prob = _prob(oracle_lib, N, 1, vn.rates(s), variant="none", bc="periodic", rho0=rho0, u0=uf,
                 rho_f=rho0, u_f=uf)
    st = oracle_lib.State(prob, np.full((1, N), rho0), uf[0], uf[1])
    st.f[:] = oracle_lib.feq(rho0, *uf)[:, None, None] + seed[:, None, :]
    r, ux, uy = st.moments()
    rest_u = (np.full_like(r, uf[0]), np.full_like(r, uf[1]))
    pot = dg.reduce_fields(r, *rest_u, rho0=rho0, u0=uf)[3]
    kin = dg.reduce_fields(np.zeros_like(r), ux, uy, rho0=rho0, u0=uf)[3]
    e0 = dg.reduce_fields(r, ux, uy, rho0=rho0, u0=uf)[3]
    assert abs(pot / kin - 1) < 5e-3, (pot, kin)
    assert e0 == pytest.approx(pot + kin, rel=1e-12)
    st.run(2 * N)
    e1 = dg.reduce_fields(*st.moments(), rho0=rho0, u0=uf)[3]
    assert e1 / e0 == pytest.approx(abs(lam[idx]) ** (4 * N), rel=1e-7)


def test_orszag_profile_normalisation():
    """Eq. (normalizedsigma): sigma~ vanishes at x0 and L and peaks at 1 at 0.8."""
    rows = dict((r[0], float(r[1])) for r in golden_rows("normalized_sigma.txt"))
    x = np.linspace(rows["x0"], rows["L"], 100001)
    sig = 3125 * (rows["L"] - x) * (x - rows["x0"]) ** 4 / (256 * (rows["L"] - rows["x0"]) ** 5)
    assert sig[0] == 0 and sig[-1] == 0
    assert x[np.argmax(sig)] == pytest.approx(rows["argmax"], abs=1e-4)
    assert sig.max() == pytest.approx(rows["max"], abs=1e-9)
    prof = wl.orszag_profile(400, 100, 1.0)
    assert prof.max() == pytest.approx(1.0, abs=1e-3)


def test_type_I_grows_where_s_plus_chi_exceeds_two(oracle_lib):
    """Sec. 2.2.1 / Eq. (effectrelax): with s + chi > 2 the type I term is unstable;
    the 100 x 100 pulse workload (s = 1.988, chi up to 0.1) blows up while the type II
    run on the same workload stays bounded."""
    w = wl.small_pulse("I", "f64")
    r1, _, _ = _run_workload(oracle_lib, w, 300).moments()
    r2, _, _ = _run_workload(oracle_lib, w.with_(variant="II"), 300).moments()
    assert not np.all(np.isfinite(r1)) or np.abs(r1).max() > 1e3 * np.abs(r2).max()
    assert np.abs(r2).max() < 1e-3


# ---------------------------------------- the paper's strategy comparison ----

def _e_l2_history(core, variant, u0, W=40, steps=600, every=50):
    """2-D acoustic pulse of Sec. 4.1 on 200 x 200 cells (b = 1/20 of the domain =
    10 cells), layer 4b, nearly inviscid (nu = 1e-5): type II with the Orszag
    profile and chi = 4/s - 0.001, the viscosity sponge, or no layer."""
    from oracle import diagnostics as dg

    w = wl.pulse_workload(200, 200, variant="II", storage="f64", b=10.0, width=W, chi_max=0.0,
                          nu=1e-5, u0=u0)
    s = w.s[0]
    if variant == "II":
        c = wl.orszag_profile(200, W, 4 / s - 0.001)
        w = w.with_(chi_x=c, chi_y=c)
    elif variant == "viscous":
        r = wl.viscous_ramp(200, W)
        w = w.with_(variant="viscous", chi_x=r, chi_y=r)
    else:
        w = w.with_(variant="none")
    prob = core.Problem(w.nx, w.ny, w.s, variant=w.variant, u0=w.u0, u_f=w.u_f, chi_x=w.chi_x,
                        chi_y=w.chi_y)
    st = core.State(prob, *w.initial_fields())
    out = []
    for _ in range(steps // every):
        st.run(every)
        out.append(dg.e_l2(st.moments()[0]))
    return np.array(out)


@pytest.mark.parametrize("u0", [(0.0, 0.0), (0.1, 0.0)])
def test_type_II_beats_the_viscosity_sponge_and_no_layer(oracle_lib, u0):
    """Figs. n3-n6: once the pulse has reached the layer, the type II layer leaves an
    E_L2 several times below both the viscosity sponge and no layer (more than 5x
    from step 350, more than 10x at step 600), the viscosity sponge is only
    slightly better than nothing, and the type II error falls fast: over steps
    200-600 the log-log slope is -3.41 at rest and -3.68 with mean flow in this
    setup (nu = 1e-5, E_L2 every 50 steps), against the paper's exponents of
    about -3.5 and -3; held to below -3.0 (a 12 % margin on the shallower one).
    A viscosity sponge in place of the type II term gives -1.9."""
    none = _e_l2_history(oracle_lib, "none", u0)
    visc = _e_l2_history(oracle_lib, "viscous", u0)
    typ2 = _e_l2_history(oracle_lib, "II", u0)
    late = slice(6, None)  # steps 350..600
    assert np.all(typ2[late] < 0.2 * visc[late]) and np.all(typ2[late] < 0.2 * none[late])
    assert typ2[-1] < 0.1 * visc[-1] and typ2[-1] < 0.1 * none[-1]
    assert np.all(visc[3:] < none[3:]) and np.all(visc[3:] > 0.5 * none[3:])
    t = np.arange(1, len(typ2) + 1) * 50.0
    sel = (t >= 200) & (t <= 600)
    slope = np.polyfit(np.log(t[sel]), np.log(typ2[sel]), 1)[0]
    assert slope < -3.0, slope
