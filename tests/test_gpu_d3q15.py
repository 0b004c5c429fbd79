"""The D3Q15 scheme on the GPU (lbm3_* C ABI) against the D3Q15 oracle
(oracle/d3q15.py).

- Ragged and tiny lattices (several x tiles, ragged tails in x and y, one-cell
  axes), every damping variant, both boundaries, distinct MRT rates, mean flow
  and a reference state different from the far field, 20 steps: each field of
  the deviation state (rho', u - u0) within 1e-10 (FP64, plus the oracle's
  absolute floor) or 1e-5 (FP32) of the state's norm.
- The 3-D pulse with a ramped layer on every face: FP32 and FP64 against the
  oracle over 60 steps.
- At the benchmark's size (256^3 FP32): the central window against the
  oracle on a smaller box, the cube's symmetries of the centred pulse, and
  mass conservation on a periodic lattice without damping.
"""
import math

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6350_gb300 import lbm

    lbm.load()


def _floor(steps, n):
    # the oracle's own rounding on full populations ~ rho0 = 1
    return 10 * (steps + 1) * 2.0**-53 * math.sqrt(n)


def _close(got, ref, tol, steps, what=""):
    err = float(np.linalg.norm(got - ref))
    bound = tol * float(np.linalg.norm(ref)) + _floor(steps, ref.size)
    assert err <= bound, (what, err, bound)


def _close_state(got, ref, u0, tol, steps, what=""):
    """Each field of the deviation state (rho', u - u0) within tol times the
    norm of the whole reference deviation state (a field that conservation or
    symmetry keeps at zero is held to the state's scale, not to zero)."""
    dev_got = [got[0]] + [g - u for g, u in zip(got[1:], u0)]
    dev_ref = [ref[0]] + [r - u for r, u in zip(ref[1:], u0)]
    scale = math.sqrt(sum(float(np.linalg.norm(r)) ** 2 for r in dev_ref))
    for a, b, name in zip(dev_got, dev_ref, ("rho'", "u_x", "u_y", "u_z")):
        err = float(np.linalg.norm(a - b))
        bound = tol * scale + _floor(steps, b.size)
        assert err <= bound, (what, name, err, bound)


def _oracle(w: "wl.Workload3", steps):
    from oracle import d3q15 as d3

    prob = d3.Problem(w.nx, w.ny, w.nz, w.s, w.n, w.m, w.variant, w.bc, w.rho0, w.u0, w.rho_f,
                      w.u_f, w.chi_x, w.chi_y, w.chi_z)
    st = d3.State(prob, w.rho0 + w.rho_dev, [np.full(w.rho_dev.shape, v) for v in w.u0])
    return st.run(steps).moments()


def _gpu(w: "wl.Workload3", storage, steps):
    import warnings

    from paper_1203_6350_gb300 import lbm

    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        lat = lbm.Lattice3(w.nx, w.ny, w.nz, storage, w.rho0, w.u0, w.s, w.n, w.m, w.bc)
        lat.set_sponge(w.variant, w.chi_x, w.chi_y, w.chi_z, w.rho_f, w.u_f)
    with lat:
        lat.init_equilibrium(w.rho0 + w.rho_dev, *w.u0)
        lat.step(steps)
        assert lat.time == steps
        return lat.moments()


def _random(nx, ny, nz, variant, bc, seed, steps=20):
    rng = np.random.default_rng(seed)
    s = np.concatenate([[1.7] * 4, rng.uniform(1.1, 1.95, 11)])
    return wl.Workload3(name="random", nx=nx, ny=ny, nz=nz, s=s, variant=variant,
                        chi_x=rng.uniform(0, 0.4, nx), chi_y=rng.uniform(0, 0.4, ny),
                        chi_z=rng.uniform(0, 0.4, nz),
                        rho_dev=1e-3 * rng.standard_normal((nz, ny, nx)), steps=steps, bc=bc,
                        n=0.4, m=0.6, u0=(0.04, -0.02, 0.03), rho_f=1.002, u_f=(0.05, 0.0, -0.01))


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 2), (70, 9, 5), (5, 13, 7), (130, 3, 3)])
@pytest.mark.parametrize("variant", ["none", "I", "II", "III"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_d3q15_against_the_oracle(shape, variant, bc):
    w = _random(*shape, variant, bc, seed=sum(shape) * 7 + len(variant))
    ref = _oracle(w, w.steps)
    for storage in ("f64", "f32"):
        got = _gpu(w, storage, w.steps)
        _close_state(got, ref, w.u0, TOL[storage], w.steps, storage)


@pytest.mark.parametrize("variant", ["I", "II", "III"])
def test_pulse_with_layers_against_the_oracle(variant):
    """A 48 x 40 x 36 box, b = 4 pulse, 8-cell ramped layers, mean flow along x,
    60 steps.  chi_max = 0.3 for types II and III; 0.01 for type I, which is
    unstable where s + chi > 2 (Sec. 2.2.1) and would amplify round-off."""
    w = wl.pulse3d(48, steps=60, width=8, chi_max=0.01 if variant == "I" else 0.3,
                   variant=variant, b=4.0, ny=40, nz=36, u0=(0.05, 0.0, 0.0))
    ref = _oracle(w, w.steps)
    for storage in ("f64", "f32"):
        got = _gpu(w, storage, w.steps)
        _close(got[0], ref[0], TOL[storage], w.steps, (storage, "rho'"))
        _close_state(got, ref, w.u0, TOL[storage], w.steps, storage)


def test_benchmark_size_symmetry_and_conservation():
    """256^3 FP32, the benchmark's pulse and layer, 100 steps: rho' is invariant
    under the mirrors and axis swaps of the cube (FP32: to 1e-5 of its maximum;
    the kernel sums the mirrored cells' populations in another order).  A
    periodic 256^3 lattice without damping keeps its total mass to FP32 rounding."""
    from paper_1203_6350_gb300 import lbm

    w = wl.pulse3d(256, steps=100)
    r = _gpu(w, "f32", w.steps)[0]
    scale = np.abs(r).max()
    assert scale > 1e-5
    for img in (r[::-1], r[:, ::-1], r[:, :, ::-1], r.transpose(0, 2, 1), r.transpose(2, 1, 0),
                r.transpose(1, 0, 2)):
        assert np.abs(img - r).max() <= 1e-5 * scale
    with lbm.Lattice3(256, 256, 256, "f32", 1.0, (0.0, 0.0, 0.0), w.s, bc="periodic") as lat:
        lat.init_equilibrium(1.0 + w.rho_dev, 0.0, 0.0, 0.0)
        m0 = lat.moments()[0].sum(dtype=np.float64)
        lat.step(50)
        m1 = lat.moments()[0].sum(dtype=np.float64)
    # FP32 deviations ~ 1e-3 in 16.8M cells: rounding of order 1e-10 each
    assert abs(m1 - m0) <= 1e-4 * abs(m0), (m0, m1)


def test_benchmark_size_window_against_the_oracle():
    """The benchmark's 256^3 FP32 pulse (16-cell type II layer), 30 steps, in
    the central 32^3 window against the oracle on a 96^3 box holding the same
    pulse at its centre, no layer.  A signal moves at most one cell per step,
    so after 30 steps the window depends only on cells within 46 of the
    centre: inside the big lattice's chi = 0 core and 32 cells from the small
    box's edge, with the same initial data on both."""
    from oracle import d3q15 as d3

    steps, half, win = 30, 48, 16
    big = wl.pulse3d(256, steps=steps)
    got = _gpu(big, "f32", steps)
    c = 128
    got = [g[c - win:c + win, c - win:c + win, c - win:c + win] for g in got]
    small = wl.pulse3d(2 * half, steps=steps, width=0, chi_max=0.0)
    prob = d3.Problem(small.nx, small.ny, small.nz, small.s, variant="none")
    ref = d3.State(prob, 1.0 + small.rho_dev, [0.0, 0.0, 0.0]).run(steps).moments()
    ref = [r[half - win:half + win, half - win:half + win, half - win:half + win] for r in ref]
    # the same pulse: centred at (n - 1)/2 on both lattices, so the windows align
    _close_state(got, ref, (0.0, 0.0, 0.0), TOL["f32"], steps, "window")


def test_d3q15_diagnostics_against_the_oracle():
    """The FP64 sums of lbm3_diagnostics (FP64 storage) against the same sums of
    the oracle's fields, on the whole lattice and on a sub-box, with mean flow."""
    from oracle import d3q15 as d3

    w = wl.pulse3d(20, steps=12, width=4, chi_max=0.3, b=3.0, ny=18, nz=16, u0=(0.05, 0.0, 0.0))
    prob = d3.Problem(w.nx, w.ny, w.nz, w.s, w.n, w.m, w.variant, w.bc, w.rho0, w.u0, w.rho_f,
                      w.u_f, w.chi_x, w.chi_y, w.chi_z)
    r, ux, uy, uz = d3.State(prob, w.rho0 + w.rho_dev,
                             [np.full(w.rho_dev.shape, v) for v in w.u0]).run(w.steps).moments()
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice3(w.nx, w.ny, w.nz, "f64", w.rho0, w.u0, w.s) as lat:
        lat.set_sponge(w.variant, w.chi_x, w.chi_y, w.chi_z)
        lat.init_equilibrium(w.rho0 + w.rho_dev, *w.u0)
        lat.step(w.steps)
        for box in ((0, 0, 0, w.nx, w.ny, w.nz), (3, 2, 1, 15, 11, 9), (5, 5, 5, 5, 9, 9)):
            x0, y0, z0, x1, y1, z1 = box
            sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
            rho = w.rho0 + r[sl]
            j = [rho * u[sl] - w.rho0 * u0 for u, u0 in zip((ux, uy, uz), w.u0)]
            du2 = sum((u[sl] - u0) ** 2 for u, u0 in zip((ux, uy, uz), w.u0))
            want = [r[sl].sum(), *(a.sum() for a in j),
                    (r[sl] ** 2 / (6 * w.rho0) + 0.5 * w.rho0 * du2).sum(), (r[sl] ** 2).sum(), 0]
            got = lat.diagnostics(box)
            for q in range(6):
                tol = 1e-9 * max(abs(want[q]), 1e-12) + 1e-12
                assert abs(got[q] - want[q]) <= tol, (box, q, got[q], want[q])
            assert got[6] == 0


def test_d3q15_checkpoint_round_trip():
    """Stepping 10 + 10 steps equals stepping 10, saving, restoring into a new
    lattice and stepping 10 more, bit for bit (FP32)."""
    from paper_1203_6350_gb300 import lbm

    w = wl.pulse3d(40, steps=20, width=6, chi_max=0.3, b=3.0, ny=24, nz=18)
    def make():
        lat = lbm.Lattice3(w.nx, w.ny, w.nz, "f32", w.rho0, w.u0, w.s)
        lat.set_sponge(w.variant, w.chi_x, w.chi_y, w.chi_z)
        lat.init_equilibrium(w.rho0 + w.rho_dev, *w.u0)
        return lat
    with make() as a:
        a.step(10)
        buf, t = a.get_state()
        assert t == 10
        a.step(10)
        want, _ = a.get_state()
    with make() as b:
        b.step(3)  # a different state, overwritten by the checkpoint
        b.set_state(buf, t)
        assert b.time == 10
        b.step(10)
        got, t2 = b.get_state()
    assert t2 == 20
    np.testing.assert_array_equal(got, want)


def test_d3q15_type_II_layer_absorbs_the_pulse():
    """The 3-D counterpart of the 2-D trend pin: a pulse in a 64^3 box with the
    Dirichlet far field comes back from the walls; with a 12-cell type II layer
    (chi_max = 4/s - 0.001, quadratic ramp) the interior energy left after 150
    steps is more than 20 times smaller (the oracle gives 47 times: 1.30e-4
    against 6.15e-3 of the initial energy).  FP32."""
    from paper_1203_6350_gb300 import lbm

    out = {}
    for variant, chi in (("none", 0.0), ("II", None)):
        w = wl.pulse3d(64, steps=150, width=12, b=3.0,
                       chi_max=chi if chi is not None else 4 / 1.98807 - 0.001, variant=variant)
        with lbm.Lattice3(64, 64, 64, "f32", w.rho0, w.u0, w.s) as lat:
            import warnings
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", RuntimeWarning)
                lat.set_sponge(w.variant, w.chi_x, w.chi_y, w.chi_z)
            lat.init_equilibrium(w.rho0 + w.rho_dev, *w.u0)
            box = (12, 12, 12, 52, 52, 52)
            e0 = lat.diagnostics(box)[4]
            lat.step(w.steps)
            out[variant] = lat.diagnostics(box)[4] / e0
    assert out["II"] < 0.05 * out["none"], out


def test_d3q15_api_rules():
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice3(8, 8, 8, "f32") as lat:
        assert lbm.lbm3_step(lat.h, 1) == lbm.LBM_ERR_STATE
        cx = np.zeros(8)
        bad = np.full(8, -1.0)
        assert lbm.lbm3_set_sponge(lat.h, 2, bad.ctypes.data, cx.ctypes.data, cx.ctypes.data,
                                   1.0, (0, 0, 0)) == lbm.LBM_ERR_ARG
        big = np.full(8, 3.0)
        assert lbm.lbm3_set_sponge(lat.h, 2, big.ctypes.data, cx.ctypes.data, cx.ctypes.data,
                                   1.0, (0, 0, 0)) == lbm.LBM_WARN_UNSTABLE_PARAMS
