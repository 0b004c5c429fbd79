"""The two-cells-per-thread step kernel against the one-cell kernel.

Both kernels evaluate the same collision in the same order, one cell per
scalar instruction or two cells per packed FP32 instruction.  The code
generator fuses some products into the adds that consume them in the packed
form and not in the scalar one, so the two agree to FP32 rounding rather
than bit for bit: after one step from the same state every stored population
agrees to a few units in the last place of the storage format, after 25 steps
the fields agree to the FP32 / 16-bit rounding level.  An indexing error
(a wrong neighbour, a lost cell, a swapped lane) would show as differences of
the size of the populations themselves.  The cases cover odd widths (the last
pair holds one cell), lattices narrower than one pair, periodic wrap, pairs
that straddle the edge of the absorbing layer and the chi = 0 rectangle.
Agreement with the FP64 oracle is covered by the parity tests, which run the
default (two-cell) kernel.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6350_gb300 import lbm

    lbm.load()


def _workload(nx, ny, bc, variant, layer, seed):
    """Random MRT rates and fields; chi either random everywhere (layer = 0) or
    a quadratic ramp of `layer` cells on every side around a chi = 0 core."""
    rng = np.random.default_rng(seed)
    if layer:
        chi_x = wl.ramp_profile(nx, layer, 0.3)
        chi_y = wl.ramp_profile(ny, layer, 0.3)
    else:
        chi_x, chi_y = rng.uniform(0, 0.5, nx), rng.uniform(0, 0.5, ny)
    return wl.Workload(name=f"pair-{nx}x{ny}", nx=nx, ny=ny,
                       s=np.array([1.6, 1.6, 1.6, 1.1, 1.2, 1.3, 1.3, 1.9, 1.9]),
                       variant=variant, bc=bc, n=0.4, m=0.6, rho0=1.0, u0=(0.04, -0.02),
                       rho_f=1.002, u_f=(0.05, -0.01), chi_x=chi_x, chi_y=chi_y,
                       rho_dev=1e-3 * rng.standard_normal((ny, nx)), steps=25, storage="f32")


def _run(w, storage, cells, steps, per_launch=1):
    """Decoded stored populations (float64, storage scale) and rho', ux, uy."""
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice.from_workload(w, storage=storage) as lat:
        lat.cells_per_thread = cells
        assert lat.cells_per_thread == cells
        lat.steps_per_launch = per_launch
        assert lat.steps_per_launch == per_launch
        lat.step(steps)
        buf, t = lat.get_state()
        assert t == steps
        fields = lat.moments()
    if storage == "f32":
        pops = buf.view(np.float32).astype(np.float64)
    elif storage == "f16dev":
        pops = buf.view(np.float16).astype(np.float64)
    else:  # bf16: the upper half of an FP32 word
        pops = (buf.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return pops, fields


# after one step: stored values within a few units in the last place of the
# format at the largest magnitude; after 25 steps: relative L2 of the fields
ONE_STEP = {"f32": 2.0**-21, "f16dev": 2.0**-9, "bf16dev": 2.0**-6}
MANY_STEPS = {"f32": 2e-5, "f16dev": 2e-3, "bf16dev": 2e-2}
# Two steps per launch keep the intermediate time level in FP32, so with 16-bit
# storage the two paths round at different steps: after 25 steps they differ
# by a random walk of ~12 roundings of 2^-11 (FP16) or 2^-8 (BF16), amplified
# where type I has s + chi > 2 (up to ~9 % per step); held to sixteen
# roundings' worth (a BF16 type I case measured ten).
MANY_STEPS_TB = {"f32": 2e-5, "f16dev": 16 * 2.0**-11, "bf16dev": 16 * 2.0**-8}


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (2, 7), (130, 3), (257, 129), (33, 64),
                                   (1025, 40)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("variant", ["none", "I", "II", "III", "viscous"])
def test_pair_kernel_matches_the_one_cell_kernel(shape, bc, variant):
    nx, ny = shape
    for layer in (0, 5):
        if layer and 2 * layer >= min(nx, ny):
            continue
        w = _workload(nx, ny, bc, variant, layer, seed=nx * 7919 + ny)
        for storage in ("f32", "f16dev", "bf16dev"):
            a, _ = _run(w, storage, 1, 1)
            b, _ = _run(w, storage, 2, 1)
            scale = np.abs(a).max()
            assert np.abs(a - b).max() <= ONE_STEP[storage] * scale, (storage, layer)
            _, fa = _run(w, storage, 1, w.steps)
            _, fb = _run(w, storage, 2, w.steps)
            for x, y in zip(fa, fb):
                den = np.linalg.norm(x)
                if den > 0:
                    assert np.linalg.norm(x - y) <= MANY_STEPS[storage] * den, (storage, layer)


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (2, 7), (130, 3), (257, 129), (64, 16),
                                   (65, 17), (129, 33), (1025, 40)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("variant", ["none", "I", "II", "III", "viscous"])
def test_two_steps_per_launch_match_one(shape, bc, variant):
    """Temporal blocking: one launch of the two-step kernel against two
    launches of the two-cell kernel (tiles of 64 x 16 cells whose ring of
    step-one cells crosses the lattice edge, wraps, or stays inside), then
    25 steps (12 two-step launches and one one-step launch).  With 16-bit
    storage one two-step launch rounds to the format once, two launches twice
    (MANY_STEPS_TB).  Type I here has s + chi up to 2.4 (rates 1.9, chi up to
    0.5): it amplifies any rounding difference without bound (Eq. effectrelax,
    reading C15), so its two 16-bit paths, which round at different steps, are
    compared after one launch only."""
    nx, ny = shape
    for layer in (0, 5):
        if layer and 2 * layer >= min(nx, ny):
            continue
        w = _workload(nx, ny, bc, variant, layer, seed=nx * 104729 + ny)
        for storage in ("f32", "f16dev", "bf16dev"):
            a, _ = _run(w, storage, 2, 2, per_launch=1)
            b, _ = _run(w, storage, 2, 2, per_launch=2)
            scale = np.abs(a).max()
            assert np.abs(a - b).max() <= 2 * ONE_STEP[storage] * scale, (storage, layer)
            if variant == "I" and storage != "f32":
                continue
            _, fa = _run(w, storage, 2, w.steps, per_launch=1)
            _, fb = _run(w, storage, 2, w.steps, per_launch=2)
            for x, y in zip(fa, fb):
                den = np.linalg.norm(x)
                if den > 0:
                    assert np.linalg.norm(x - y) <= MANY_STEPS_TB[storage] * den, (storage, layer)


def test_two_steps_per_launch_through_graph_chunks():
    """70 steps: one replayed graph of 32 two-step launches, then three more;
    against the one-step-per-launch run, and the step counter."""
    from paper_1203_6350_gb300 import lbm

    w = _workload(300, 190, "dirichlet", "III", 16, seed=11)
    _, fa = _run(w, "f32", 2, 70, per_launch=1)
    _, fb = _run(w, "f32", 2, 70, per_launch=2)
    for x, y in zip(fa, fb):
        assert np.linalg.norm(x - y) <= MANY_STEPS["f32"] * np.linalg.norm(x)
    with lbm.Lattice.from_workload(w, storage="f32") as lat:
        lat.steps_per_launch = 2
        lat.step(70)
        assert lat.time == 70
        lat.step(1)
        assert lat.time == 71


def test_kernel_switches_rebuild_the_captured_graphs():
    """A handle switched between the kernels mid-run (64-step graphs are
    captured on both sides of each switch) continues with the kernel it was
    switched to: each segment equals, bit for bit, the same kernel run from
    the segment's starting state on a fresh handle."""
    from paper_1203_6350_gb300 import lbm

    w = _workload(301, 200, "dirichlet", "II", 16, seed=5)
    with lbm.Lattice.from_workload(w, storage="f32") as lat:
        lat.cells_per_thread = 2
        lat.step(70)
        mid, _ = lat.get_state()
        lat.cells_per_thread = 1
        lat.step(65)
        got1, t1 = lat.get_state()
        lat.cells_per_thread = 2
        lat.step(65)
        got2, t2 = lat.get_state()
    assert (t1, t2) == (135, 200)
    for start, t0, cells, want in ((mid, 70, 1, got1), (got1, 135, 2, got2)):
        with lbm.Lattice.from_workload(w, storage="f32") as ref:
            ref.cells_per_thread = cells
            ref.set_state(start, t0)
            ref.step(65)
            b, t = ref.get_state()
        assert t == t0 + 65
        assert b.tobytes() == want.tobytes(), cells


def test_cells_per_thread_choices():
    from paper_1203_6350_gb300 import lbm

    w = _workload(40, 30, "dirichlet", "II", 5, seed=1)
    with lbm.Lattice.from_workload(w, storage="f64") as lat:
        assert lat.cells_per_thread == 1
        assert lbm.lbm_set_cells_per_thread(lat.h, 2) == lbm.LBM_ERR_ARG
        assert lat.cells_per_thread == 1
    with lbm.Lattice.from_workload(w, storage="f32") as lat:
        assert lat.cells_per_thread == 2  # the default where available
        for bad in (0, 3, -1):
            assert lbm.lbm_set_cells_per_thread(lat.h, bad) == lbm.LBM_ERR_ARG
            assert lbm.lbm_set_steps_per_launch(lat.h, bad) == lbm.LBM_ERR_ARG
        assert lat.cells_per_thread == 2
        lat.steps_per_launch = 2
        lat.cells_per_thread = 1  # falls back to one step per launch
        assert lat.steps_per_launch == 1
        assert lbm.lbm_set_steps_per_launch(lat.h, 2) == lbm.LBM_ERR_ARG
    with lbm.Lattice.from_workload(w, storage="f64") as lat:
        assert lbm.lbm_set_steps_per_launch(lat.h, 2) == lbm.LBM_ERR_ARG
        assert lat.steps_per_launch == 1
