"""The two-step kernel with TMA-staged input (FP32, FP16 and BF16 storage,
Dirichlet) against the same two-step arithmetic on plain loads: bit-identical stored states on
ragged, tiny and large lattices, every damping variant, odd step counts (the
one-step remainder) and graph-replayed chunks; where it is available.
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


def _state(w, tma, steps, chunks=None, storage="f32"):
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice.from_workload(w, storage=storage) as lat:
        lat.cells_per_thread = 2
        lat.steps_per_launch = 2
        lat.tma_staging = tma
        assert lat.tma_staging == tma
        for n in (chunks or [steps]):
            lat.step(n)
        buf, t = lat.get_state()
        assert t == steps
        return buf


def _random(nx, ny, variant, seed, steps):
    rng = np.random.default_rng(seed)
    return wl.Workload(name=f"tma-{nx}x{ny}", nx=nx, ny=ny,
                       s=np.array([1.6, 1.6, 1.6, 1.1, 1.2, 1.3, 1.3, 1.9, 1.9]),
                       variant=variant, bc="dirichlet", n=0.4, m=0.6, rho0=1.0,
                       u0=(0.04, -0.02), rho_f=1.002, u_f=(0.05, -0.01),
                       chi_x=rng.uniform(0, 0.5, nx), chi_y=rng.uniform(0, 0.5, ny),
                       rho_dev=1e-3 * rng.standard_normal((ny, nx)), steps=steps, storage="f32")


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (3, 5), (64, 16), (65, 17), (129, 33),
                                   (1025, 40), (300, 200)])
@pytest.mark.parametrize("variant", ["none", "I", "II", "III", "viscous"])
@pytest.mark.parametrize("storage", ["f32", "f16dev", "bf16dev"])
def test_tma_staging_is_bit_identical_to_plain_loads(shape, variant, storage):
    w = _random(*shape, variant, seed=shape[0] * 7 + shape[1], steps=11)
    a = _state(w, True, w.steps, storage=storage)
    b = _state(w, False, w.steps, storage=storage)
    np.testing.assert_array_equal(a, b)


def _edged(nx, ny, variant, width, seed, steps):
    """A lattice with a real bulk: chi = 0.4 (d / width)^2 in a layer `width`
    cells deep on every side and zero inside, random deviations everywhere."""
    rng = np.random.default_rng(seed)

    def ramp(n):
        i = np.arange(n)
        d = np.maximum(np.maximum(width - i, i - (n - 1 - width)), 0) / width
        return 0.4 * d * d

    return wl.Workload(name=f"edged-{nx}x{ny}", nx=nx, ny=ny,
                       s=np.array([1.6, 1.6, 1.6, 1.1, 1.2, 1.3, 1.3, 1.9, 1.9]),
                       variant=variant, bc="dirichlet", n=0.4, m=0.6, rho0=1.0,
                       u0=(0.04, -0.02), rho_f=1.002, u_f=(0.05, -0.01),
                       chi_x=ramp(nx), chi_y=ramp(ny),
                       rho_dev=1e-3 * rng.standard_normal((ny, nx)), steps=steps, storage="f32")


@pytest.mark.parametrize("variant", ["I", "II", "III", "viscous"])
@pytest.mark.parametrize("storage", ["f32", "f16dev", "bf16dev"])
def test_a_layer_edge_inside_a_warp_changes_no_bit(variant, storage):
    """The TMA kernel chooses between the bulk and the layer collision per warp,
    the plain-load two-step kernel per pair; with the edge of the bulk inside
    warps (a 37-cell layer) their stored states still agree bit for bit, since
    the layer collision at chi = 0 is the bulk collision exactly."""
    w = _edged(300, 200, variant, 37, seed=11, steps=11)
    a = _state(w, True, w.steps, storage=storage)
    b = _state(w, False, w.steps, storage=storage)
    np.testing.assert_array_equal(a, b)


def test_tma_staging_across_graph_chunks():
    """150 steps as 64 + 64 + 22: graph replays of 32 two-step launches and a
    one-step remainder."""
    w = _random(333, 97, "II", seed=5, steps=150)
    for storage in ("f32", "f16dev"):
        a = _state(w, True, w.steps, chunks=[64, 64, 22], storage=storage)
        b = _state(w, False, w.steps, chunks=[150], storage=storage)
        np.testing.assert_array_equal(a, b)


def test_tma_staging_availability():
    from paper_1203_6350_gb300 import lbm

    w = _random(64, 16, "II", seed=1, steps=2)
    with lbm.Lattice.from_workload(w, storage="f32") as lat:
        assert not lat.tma_staging  # the default only above four times L2
        lat.tma_staging = True
        assert lat.tma_staging
    with lbm.Lattice.from_workload(w.with_(bc="periodic"), storage="f32") as lat:
        assert not lat.tma_staging
        with pytest.raises(lbm.LbmError):
            lat.tma_staging = True
    with lbm.Lattice.from_workload(w, storage="f16dev") as lat:
        assert not lat.tma_staging
        assert lbm.lbm_set_tma_staging(lat.h, 1) == lbm.LBM_OK
        assert lbm.lbm_set_tma_staging(lat.h, 0) == lbm.LBM_OK
        assert lbm.lbm_set_tma_staging(lat.h, 2) == lbm.LBM_ERR_ARG
    with lbm.Lattice.from_workload(w, storage="f64") as lat:
        assert lbm.lbm_set_tma_staging(lat.h, 1) == lbm.LBM_ERR_ARG


def test_tma_staging_at_2048_is_bit_identical_to_plain_loads():
    """The 2048^2 pulse with its 128-cell layer, 200 steps of two steps per
    launch (the library's default there, with plain loads: the configuration
    whose result test_gpu_parity holds to 1e-5 of the oracle), against TMA
    staging."""
    from paper_1203_6350_gb300 import lbm

    w = wl.quiescent(2048, storage="f32", steps=200, pulse=True)
    states = []
    for tma in (True, False):
        with lbm.Lattice.from_workload(w) as lat:
            assert lat.steps_per_launch == 2 and not lat.tma_staging
            lat.tma_staging = tma
            lat.step(w.steps)
            states.append(lat.get_state()[0])
    np.testing.assert_array_equal(states[0], states[1])


def test_tma_staging_is_the_default_at_4096_and_matches_plain_loads():
    """4096^2 (1.2 GB of state, above four times L2): TMA staging by default,
    20 steps bit-identical to plain loads; the quiescent lattice stays exactly
    at rest."""
    from paper_1203_6350_gb300 import lbm

    w = wl.quiescent(4096, storage="f32", steps=20, pulse=True)
    states = []
    for tma in (None, False):
        with lbm.Lattice.from_workload(w) as lat:
            if tma is None:
                assert lat.steps_per_launch == 2 and lat.tma_staging
            else:
                lat.tma_staging = tma
            lat.step(w.steps)
            states.append(lat.get_state()[0])
    np.testing.assert_array_equal(states[0], states[1])


def test_tma_staging_in_batches_is_bit_identical(monkeypatch):
    """A batch of mixed lattices (Dirichlet and periodic, every variant, odd
    budgets that end on a one-step launch, 131 steps) with two steps per launch:
    TMA-staged input for the Dirichlet instances (the FP32 default) against
    plain loads, bit for bit."""
    from test_gpu_batch import _mixed_workloads

    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch

    works = _mixed_workloads("f32")
    out = []
    for env in (None, "0"):
        if env is None:
            monkeypatch.delenv("LBM_BATCH_TMA", raising=False)
        else:
            monkeypatch.setenv("LBM_BATCH_TMA", env)
        with Batch("f32") as b:
            assert lbm.lbm_batch_tma_staging(b.b) == (1 if env is None else 0)
            b.cells_per_thread = 2
            b.steps_per_launch = 2
            ids = [b.add_workload(w) for w in works]
            b.step(131)
            out.append([b.moments(i) for i in ids])
    for a, c in zip(*out):
        for x, y in zip(a, c):
            np.testing.assert_array_equal(x, y)


# ------------------------------------------ the bounded wait's give-up path ----
#
# LBM_TMA_WAIT_POLLS=0 at set-up makes each tile's wait for its staged copy
# give up before its first poll.  Every copy is still real and in bounds, so
# nothing fails on the device: the CTA votes to stop, thread 0 waits for the
# copy in flight (full bound) and raises the error flag, and the CTA returns.
# The host must then report LBM_ERR_CUDA and the context must stay usable.


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_a_wait_that_gives_up_is_reported_single_lattice(monkeypatch, storage):
    from paper_1203_6350_gb300 import lbm

    w = _random(300, 200, "II", seed=5, steps=6)
    monkeypatch.setenv("LBM_TMA_WAIT_POLLS", "0")
    lat = lbm.Lattice.from_workload(w, storage=storage)
    try:
        lat.cells_per_thread = 2
        lat.steps_per_launch = 2
        lat.tma_staging = True
        monkeypatch.delenv("LBM_TMA_WAIT_POLLS")
        lat.step(w.steps)
        with pytest.raises(lbm.LbmError) as e:
            lat.moments()
        assert e.value.code == lbm.LBM_ERR_CUDA and "TMA" in str(e.value)
    finally:
        lat.close()
    # the context survived: a new lattice gives the plain-load result
    np.testing.assert_array_equal(_state(w, True, w.steps, storage=storage),
                                  _state(w, False, w.steps, storage=storage))


def test_a_wait_that_gives_up_is_reported_batch(monkeypatch):
    from paper_1203_6350_gb300 import lbm
    from paper_1203_6350_gb300.batch import Batch

    w = _random(130, 70, "III", seed=9, steps=8)
    monkeypatch.setenv("LBM_TMA_WAIT_POLLS", "0")
    with Batch("f32") as bt:
        monkeypatch.delenv("LBM_TMA_WAIT_POLLS")
        bt.configure(2, 2, (64, 16))
        assert lbm.lbm_batch_tma_staging(bt.b) == 1
        i = bt.add_workload(w)
        bt.step(w.steps)
        with pytest.raises(lbm.LbmError) as e:
            bt.moments(i)
        assert e.value.code == lbm.LBM_ERR_CUDA and "TMA" in str(e.value)
    with Batch("f32") as bt:
        bt.configure(2, 2, (64, 16))
        i = bt.add_workload(w)
        bt.step(w.steps)
        got = bt.moments(i)[0]
    from helpers import run_oracle
    ref = run_oracle(w)[0]
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
