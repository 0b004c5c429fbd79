"""Batched stepping (lbm_batch_*): each lattice in a batch must give the result
of the single-lattice path, whatever else is in the batch, whatever the tile
shape, and whenever it was admitted.

Within the batched path the per-cell instruction sequence does not depend on
the tile shape or on the other instances, so those comparisons are bit-exact,
for the one-cell and for the two-cell (packed FP32) batched kernel alike.
Against the single-lattice kernel the source arithmetic is shared but the
compiler may contract multiply-adds differently in the two kernels: FP64 is
bit-exact there, FP32 / FP16 agree to a few ulps (held to the parity
tolerances)."""
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


def _mixed_workloads(storage):
    rng = np.random.default_rng(11)
    mrt = np.array([1.7, 1.7, 1.7, 1.2, 1.4, 1.6, 1.6, 1.9, 1.9])
    out = []
    shapes = [(37, 53), (130, 64), (64, 257), (1, 1), (200, 9), (96, 96)]
    variants = ["none", "I", "II", "III", "II", "III"]
    for k, ((nx, ny), var) in enumerate(zip(shapes, variants)):
        w = wl.pulse_workload(nx, ny, variant=var, storage=storage, eps=1e-3, b=3.0,
                              width=max(0, min(nx, ny) // 5),
                              # type I stays stable only while s + chi <= 2 (Eq. effectrelax)
                              chi_max=0.08 if var == "I" else 0.3,
                              u0=(0.04 * (k % 3), 0.01), steps=40 + 17 * k,
                              bc="periodic" if k % 2 else "dirichlet", name=f"mix-{k}")
        if k % 2:
            w = w.with_(s=mrt)
        if nx * ny > 1:
            w = w.with_(rho_dev=1e-3 * rng.standard_normal((ny, nx)))
        out.append(w)
    return out


TOL = {"f64": 1e-12, "f32": 1e-5, "f16dev": 1e-2}


def _close(a, b, tol):
    if tol == 0:
        np.testing.assert_array_equal(a, b)
        return
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    if fin.any():
        assert np.linalg.norm(a[fin] - b[fin]) <= tol * np.linalg.norm(b[fin]) + 1e-300


def _single(w, storage, steps):
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice.from_workload(w, storage=storage) as lat:
        lat.step(steps)
        return lat.moments()


@pytest.mark.parametrize("storage", ["f32", "f64", "f16dev"])
def test_batch_equals_single_lattice(storage):
    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads(storage)
    with Batch(storage) as b:
        ids = [b.add_workload(w) for w in works]
        b.step(max(w.steps for w in works) + 5)
        for i, w in zip(ids, works):
            assert b.time(i) == w.steps
            got = b.moments(i)
            want = _single(w, storage, w.steps)
            for a, c in zip(got, want):
                _close(a, c, 0 if storage == "f64" else TOL[storage])


def _batch_run(works, storage, tiling=None, steps=100, cells=None, per_launch=None):
    from paper_1203_6350_gb300.batch import Batch

    with Batch(storage, tiling=tiling) as b:
        if cells is not None:
            b.cells_per_thread = cells
            assert b.cells_per_thread == cells
        if per_launch is not None:
            b.steps_per_launch = per_launch
            assert b.steps_per_launch == per_launch
        ids = [b.add_workload(w) for w in works]
        b.step(steps)
        return [b.moments(i)[0] for i in ids]


@pytest.mark.parametrize("cells", [1, 2])
@pytest.mark.parametrize("tiling", [(32, 8), (64, 4), (128, 2), (128, 16), (256, 1), (256, 4)])
def test_tile_shape_does_not_change_results(tiling, cells):
    works = _mixed_workloads("f32")
    ref = _batch_run(works, "f32", cells=cells)
    for r, q in zip(_batch_run(works, "f32", tiling, cells=cells), ref):
        np.testing.assert_array_equal(r, q)


@pytest.mark.parametrize("cells", [1, 2])
def test_result_alone_equals_result_in_the_mix(cells):
    works = _mixed_workloads("f32")
    mixed = _batch_run(works, "f32", cells=cells)
    for w, m in zip(works, mixed):
        (alone,) = _batch_run([w], "f32", cells=cells)
        np.testing.assert_array_equal(alone, m)


@pytest.mark.parametrize("storage", ["f32", "f16dev", "bf16dev"])
def test_pair_batch_kernel_matches_the_one_cell_batch_kernel(storage):
    """The two batched kernels agree to the storage format's rounding level
    (the pair form's fused products differ in the last bits; see
    test_gpu_pair.py) on ragged, 1-cell, periodic, MRT and layered lattices."""
    works = _mixed_workloads(storage)
    tol = {"f32": 1e-5, "f16dev": 1e-2, "bf16dev": 6e-2}[storage]
    one = _batch_run(works, storage, cells=1)
    two = _batch_run(works, storage, cells=2)
    for a, c in zip(two, one):
        _close(a, c, tol)


def test_cells_per_thread_of_a_batch():
    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch

    with Batch("f64") as b:
        assert b.cells_per_thread == 1
        assert lbm.lbm_batch_set_cells_per_thread(b.b, 2) == lbm.LBM_ERR_ARG
    with Batch("f16dev") as b:
        assert b.cells_per_thread == 2
    with Batch("f32") as b:
        assert b.cells_per_thread == 1
        for bad in (0, 3):
            assert lbm.lbm_batch_set_cells_per_thread(b.b, bad) == lbm.LBM_ERR_ARG
        b.cells_per_thread = 2
        assert b.cells_per_thread == 2


def test_staggered_admission_and_removal():
    """Instances admitted at different global steps, with different budgets,
    including one added while another is mid-run and one removed early."""
    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads("f32")
    with Batch("f32") as b:
        a = b.add_workload(works[2].with_(steps=90))
        b.step(21)
        c = b.add_workload(works[5].with_(steps=50))
        d = b.add_workload(works[0].with_(steps=200))
        b.step(33)  # 32-step graph chunk + 1 direct step
        b.remove(d)
        e = b.add_workload(works[1].with_(steps=7))
        b.step(64)
        assert b.time(a) == 90 and b.time(c) == 50 and b.time(e) == 7
        for i, w, n in ((a, works[2], 90), (c, works[5], 50), (e, works[1], 7)):
            _close(b.moments(i)[0], _single(w, "f32", n)[0], TOL["f32"])
            (alone,) = _batch_run([w.with_(steps=n)], "f32", steps=n + 3)
            np.testing.assert_array_equal(b.moments(i)[0], alone)
        assert len(b) == 3


def test_batch_against_the_oracle():
    from helpers import rel_l2, run_oracle
    from paper_1203_6350_gb300.batch import Batch

    w = wl.small_pulse("II", "f64")
    with Batch("f64") as b:
        i = b.add_workload(w.with_(steps=120))
        b.step(200)
        got = b.moments(i)[0]
    ref = run_oracle(w, 120)[0]
    # 1e-10 relative plus the oracle's own FP64 rounding (~10 x 2^-53 per cell per step)
    floor = 10 * 121 * 2.0**-53 * np.sqrt(ref.size)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref) + floor, rel_l2(got, ref)


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_two_steps_per_batched_launch(storage):
    """Temporal blocking in the batch: budgets of 40, 57, 74, 91, 108 and 125
    steps (odd budgets end on a one-step half of a two-step launch), stepped
    131 steps (four 32-step graphs, one two-step and one one-step launch),
    against one step per launch at the format's rounding level, and the step
    counters."""
    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads(storage)
    tol = {"f32": 1e-5, "f16dev": 1e-2}[storage]
    one = _batch_run(works, storage, steps=131, cells=2, per_launch=1)
    two = _batch_run(works, storage, steps=131, cells=2, per_launch=2)
    for a, c in zip(two, one):
        _close(a, c, tol)
    with Batch(storage) as b:
        b.cells_per_thread = 2
        b.steps_per_launch = 2
        ids = [b.add_workload(w) for w in works]
        b.step(131)
        for i, w in zip(ids, works):
            assert b.time(i) == w.steps


def test_two_step_batch_alone_equals_in_the_mix_and_staggered():
    """Two-step launches: a lattice alone and in the mix are bit-identical;
    instances admitted mid-run, at odd global steps, with odd budgets, end with
    the single-lattice result (rounding level) and their own step counts."""
    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads("f32")
    mixed = _batch_run(works, "f32", cells=2, per_launch=2)
    for w, m in zip(works, mixed):
        (alone,) = _batch_run([w], "f32", cells=2, per_launch=2)
        np.testing.assert_array_equal(alone, m)
    with Batch("f32") as b:
        b.cells_per_thread = 2
        b.steps_per_launch = 2
        a = b.add_workload(works[2].with_(steps=91))
        b.step(21)  # ends on a one-step launch: the global step is now odd
        c = b.add_workload(works[5].with_(steps=51))
        d = b.add_workload(works[0].with_(steps=200))
        b.step(33)
        b.remove(d)
        e = b.add_workload(works[1].with_(steps=7))
        b.step(65)
        assert b.time(a) == 91 and b.time(c) == 51 and b.time(e) == 7
        for i, w, n in ((a, works[2], 91), (c, works[5], 51), (e, works[1], 7)):
            _close(b.moments(i)[0], _single(w, "f32", n)[0], TOL["f32"])


def test_steps_per_launch_of_a_batch():
    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch

    with Batch("f32") as b:
        assert b.steps_per_launch == 1
        assert lbm.lbm_batch_set_steps_per_launch(b.b, 2) == lbm.LBM_ERR_ARG  # needs pairs
        b.cells_per_thread = 2
        b.steps_per_launch = 2
        assert b.steps_per_launch == 2
        b.cells_per_thread = 1
        assert b.steps_per_launch == 1
        for bad in (0, 3):
            assert lbm.lbm_batch_set_steps_per_launch(b.b, bad) == lbm.LBM_ERR_ARG
    with Batch("f64") as b:
        assert lbm.lbm_batch_set_steps_per_launch(b.b, 2) == lbm.LBM_ERR_ARG


def test_autotuner_picks_a_kernel_and_tile(tmp_path, monkeypatch):
    """The autotuner times every (cells per thread, steps per launch, tile)
    configuration on the shape set, caches the fastest, and a batch built from
    it steps to the same result as the default batch (rounding level)."""
    from paper_1203_6350_gb300 import autotune

    monkeypatch.setenv("LBM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    works = _mixed_workloads("f32")
    shapes = [(w.nx, w.ny) for w in works]
    configs = [(1, 1, 64, 8), (2, 1, 128, 16), (2, 2) + autotune.TWO_STEP_TILE]
    cfg = autotune.tuned_config(shapes, "f32", configs=configs)
    assert (cfg["cells"], cfg["steps_per_launch"]) + tuple(cfg["tile"]) in configs
    assert autotune.tuned_config(shapes, "f32") == cfg  # served from the cache
    from paper_1203_6350_gb300.batch import Batch

    with Batch("f32", config=cfg) as b:
        assert b.cells_per_thread == cfg["cells"]
        assert b.steps_per_launch == cfg["steps_per_launch"]
        ids = [b.add_workload(w) for w in works]
        b.step(100)
        got = [b.moments(i)[0] for i in ids]
    for a, c in zip(got, _batch_run(works, "f32")):
        _close(a, c, TOL["f32"])
