"""Padding canaries: with LBM_CANARY=1 at creation the padding of every row of
both population buffers (elements nx .. pitch - 1) holds all-one bytes, a NaN
in every storage format.  After stepping, with every kernel the library
launches (one and two cells per thread, one and two steps per launch, TMA
staging, the batched class kernels, D3Q15), on ragged lattices whose rows end
inside a tile:
  - the padding of the raw state is still all-one bytes (no kernel wrote it);
  - the cells equal, bit for bit, those of the same run without canaries (no
    kernel read padding into a result: a NaN would have spread).
This stands in for a memory checker on the row padding, the one region inside
the allocations that no kernel may touch.
"""
import warnings

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

ES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6350_gb300 import lbm

    lbm.load()


def _split(buf, rows, nx, es):
    """(cells, padding) byte views of a raw state of `rows` rows."""
    pitch_bytes = buf.nbytes // rows
    assert pitch_bytes * rows == buf.nbytes and pitch_bytes % es == 0
    a = buf.reshape(rows, pitch_bytes)
    return a[:, : nx * es], a[:, nx * es:]


def _workload(nx, ny, variant, bc, seed, steps):
    rng = np.random.default_rng(seed)
    return wl.Workload(name=f"canary-{nx}x{ny}", nx=nx, ny=ny,
                       s=np.array([1.6, 1.6, 1.6, 1.1, 1.2, 1.3, 1.3, 1.9, 1.9]),
                       variant=variant, bc=bc, n=0.4, m=0.6, rho0=1.0, u0=(0.04, -0.02),
                       rho_f=1.002, u_f=(0.05, -0.01),
                       chi_x=rng.uniform(0, 0.08 if variant == "I" else 0.5, nx),
                       chi_y=rng.uniform(0, 0.08 if variant == "I" else 0.5, ny),
                       rho_dev=1e-3 * rng.standard_normal((ny, nx)), steps=steps,
                       storage="f32", source=(2e-3, 0.3, 0.7))


def _run(monkeypatch, canary, w, storage, cpt, spl, tma):
    from paper_1203_6350_gb300 import lbm

    if canary:
        monkeypatch.setenv("LBM_CANARY", "1")
    else:
        monkeypatch.delenv("LBM_CANARY", raising=False)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        lat = lbm.Lattice.from_workload(w, storage=storage)
    with lat:
        lat.cells_per_thread = cpt
        lat.steps_per_launch = spl
        if tma is not None:
            lat.tma_staging = tma
        lat.step(w.steps)
        buf, t = lat.get_state()
        assert t == w.steps
    return buf


# (storage, cells per thread, steps per launch, TMA staging)
KERNELS = [("f64", 1, 1, None), ("f32", 1, 1, None), ("f32", 2, 1, None), ("f32", 2, 2, False),
           ("f32", 2, 2, True), ("f16dev", 1, 1, None), ("f16dev", 2, 1, None),
           ("f16dev", 2, 2, None), ("f16dev", 2, 2, True), ("bf16dev", 2, 1, None),
           ("bf16dev", 2, 2, None), ("bf16dev", 2, 2, True)]


@pytest.mark.parametrize("kernel", KERNELS, ids=lambda k: "-".join(map(str, k)))
@pytest.mark.parametrize("bc", ["dirichlet", "periodic", "channel"])
@pytest.mark.parametrize("shape", [(1, 1), (45, 13), (131, 37), (300, 77)])
def test_no_kernel_touches_row_padding(monkeypatch, kernel, bc, shape):
    storage, cpt, spl, tma = kernel
    if bc != "dirichlet" and tma:
        pytest.skip("TMA staging is for the Dirichlet boundary")
    if bc == "channel" and spl == 2:
        pytest.skip("the channel runs one step per launch")
    nx, ny = shape
    if bc == "channel" and nx < 2:
        pytest.skip("the channel needs nx >= 2")
    variant = ["none", "I", "II", "III", "viscous"][(nx + ny) % 5]
    w = _workload(nx, ny, variant, bc, seed=nx * 31 + ny, steps=9)
    with_c = _run(monkeypatch, True, w, storage, cpt, spl, tma)
    without = _run(monkeypatch, False, w, storage, cpt, spl, tma)
    es = ES[storage]
    cells_c, pad_c = _split(with_c, 9 * ny, nx, es)
    cells, _ = _split(without, 9 * ny, nx, es)
    if pad_c.size == 0:  # nx fills whole 128-byte rows: no padding to check
        assert nx * es % 128 == 0
    assert np.all(pad_c == 0xFF), "a kernel wrote into the row padding"
    np.testing.assert_array_equal(cells_c, cells)


def test_canaries_are_painted(monkeypatch):
    """The mode is on: right after creation and initialisation the padding of
    the state reads as all-one bytes, and without the mode it reads as zero."""
    from paper_1203_6350_gb300 import lbm

    w = _workload(45, 13, "II", "dirichlet", seed=1, steps=0)
    for canary, byte in ((True, 0xFF), (False, 0x00)):
        if canary:
            monkeypatch.setenv("LBM_CANARY", "1")
        else:
            monkeypatch.delenv("LBM_CANARY", raising=False)
        with lbm.Lattice.from_workload(w) as lat:
            _, pad = _split(lat.get_state()[0], 9 * 13, 45, 4)
            assert pad.size > 0 and np.all(pad == byte)


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_batched_kernels_leave_padding_alone(monkeypatch, storage):
    """Mixed batch (every variant, Dirichlet and periodic, ragged shapes, odd
    budgets), one and two steps per launch: padding intact, cells identical
    to a batch without canaries."""
    from test_gpu_batch import _mixed_workloads

    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads(storage)
    for spl in (1, 2):
        states = []
        for canary in (True, False):
            if canary:
                monkeypatch.setenv("LBM_CANARY", "1")
            else:
                monkeypatch.delenv("LBM_CANARY", raising=False)
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", RuntimeWarning)
                with Batch(storage) as b:
                    b.cells_per_thread = 2
                    b.steps_per_launch = spl
                    ids = [b.add_workload(w) for w in works]
                    b.step(131)
                    states.append([b.get_state(i) for i in ids])
        for w, sc, s0 in zip(works, *states):
            cells_c, pad_c = _split(sc, 9 * w.ny, w.nx, ES[storage])
            cells, _ = _split(s0, 9 * w.ny, w.nx, ES[storage])
            assert np.all(pad_c == 0xFF), (w.name, spl)
            np.testing.assert_array_equal(cells_c, cells)


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_d3q15_leaves_padding_alone(monkeypatch, storage, bc):
    from paper_1203_6350_gb300 import lbm

    rng = np.random.default_rng(5)
    nx, ny, nz = 37, 11, 9
    s = np.concatenate([[1.7] * 4, rng.uniform(1.1, 1.95, 11)])
    chi = [rng.uniform(0, 0.4, n) for n in (nx, ny, nz)]
    rho = 1.0 + 1e-3 * rng.standard_normal((nz, ny, nx))
    states = []
    for canary in (True, False):
        if canary:
            monkeypatch.setenv("LBM_CANARY", "1")
        else:
            monkeypatch.delenv("LBM_CANARY", raising=False)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", RuntimeWarning)
            lat = lbm.Lattice3(nx, ny, nz, storage, 1.0, (0.03, -0.02, 0.01), s, 0.4, 0.6, bc)
            lat.set_sponge("III", *chi, 1.001, (0.03, -0.02, 0.01))
        with lat:
            lat.init_equilibrium(rho, 0.03, -0.02, 0.01)
            lat.step(7)
            states.append(lat.get_state()[0])
    es = ES[storage]
    cells_c, pad_c = _split(states[0], 15 * ny * nz, nx, es)
    cells, _ = _split(states[1], 15 * ny * nz, nx, es)
    assert pad_c.size > 0 and np.all(pad_c == 0xFF)
    np.testing.assert_array_equal(cells_c, cells)


def test_batch_get_state_arguments():
    """lbm_batch_get_state: unknown id and size mismatch are LBM_ERR_ARG, an
    instance before initialisation LBM_ERR_STATE; afterwards the raw state
    holds the initial deviations (rest state: zero cells)."""
    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch

    with Batch("f32") as b:
        i = b.add(45, 13, steps=4)
        n = lbm.lbm_batch_state_bytes(b.b, i)
        assert n == 9 * 13 * 64 * 4
        assert lbm.lbm_batch_state_bytes(b.b, 12345) == 0
        buf = np.empty(n, dtype=np.uint8)
        assert lbm.lbm_batch_get_state(b.b, i, buf.ctypes.data, n, 0) == lbm.LBM_ERR_STATE
        b.init_equilibrium(i, np.ones((13, 45)), np.zeros((13, 45)), np.zeros((13, 45)))
        assert lbm.lbm_batch_get_state(b.b, 12345, buf.ctypes.data, n, 0) == lbm.LBM_ERR_ARG
        assert lbm.lbm_batch_get_state(b.b, i, buf.ctypes.data, n - 4, 0) == lbm.LBM_ERR_ARG
        cells, _ = _split(b.get_state(i), 9 * 13, 45, 4)
        assert not cells.any()
