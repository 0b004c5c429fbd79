"""The damping strength swept toward the critical value of Eq. criticalchi, on the
CUDA path (through the C ABI) against the FP64 oracle.

Type II on the 100 x 100 pulse (20-cell quadratic ramp), chi_max = 0.1, 0.5,
1.0, 1.5, 1.9 and 4/s - 0.001.  For each strength both sides report:
  R      the interior acoustic energy after 300 steps over its initial value
         (reading C14);
  E_wall the energy of the two cells next to the wall, summed every 5 steps
         over the first 150, over the same initial value: what crossed the
         layer.
The GPU side takes every sum from the library's FP64 diagnostics
(lbm_diagnostics), the oracle side from its own fields.  Tolerances, relative
to the oracle's value: FP64 storage 1e-6 (the oracle's absolute rounding,
~1e-13 per cell after 300 steps, against ring fields of ~1e-7); FP32 storage
1e-2, below the smallest step between neighbouring strengths (6 %), so the GPU
reproduces the trend itself, which is also asserted on its own numbers.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import interior_region, oracle_problem, ring_regions

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-6, "f32": 1e-2}
EVERY, RING_STEPS, STEPS = 5, 150, 300


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6350_gb300 import lbm

    lbm.load()


def _oracle(w):
    from oracle import core
    from oracle import diagnostics as dg

    st = core.State(oracle_problem(core, w), *w.initial_fields())
    reg = interior_region(w)
    e0 = dg.reduce_fields(*st.moments(), region=reg)[3]
    wall, t = 0.0, 0
    while t < RING_STEPS:
        st.run(EVERY)
        t += EVERY
        f = st.moments()
        wall += EVERY * sum(dg.reduce_fields(*f, region=q)[3] for q in ring_regions(w.nx, w.ny))
    st.run(STEPS - t)
    return dg.reduce_fields(*st.moments(), region=reg)[3] / e0, wall / e0


def _gpu(w, storage):
    from paper_1203_6350_gb300 import lbm

    with lbm.Lattice.from_workload(w, storage=storage) as lat:
        reg = interior_region(w)
        e0 = lat.diagnostics(reg)[3]
        wall, t = 0.0, 0
        while t < RING_STEPS:
            lat.step(EVERY)
            t += EVERY
            wall += EVERY * sum(lat.diagnostics(q)[3] for q in ring_regions(w.nx, w.ny))
        lat.step(STEPS - t)
        return lat.diagnostics(reg)[3] / e0, wall / e0


_ref = {}


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_chi_sweep_against_the_oracle(storage):
    sweep = wl.chi_sweep(storage)
    if not _ref:
        _ref.update({i: _oracle(w) for i, w in enumerate(sweep)})
    got = [_gpu(w, storage) for w in sweep]
    for i, w in enumerate(sweep):
        for name, g, r in zip(("R", "E_wall"), got[i], _ref[i]):
            assert abs(g - r) <= TOL[storage] * abs(r), (storage, w.chi_max, name, g, r)
    wall = np.array([g[1] for g in got])
    assert wall[0] > 1e4 * wall[1] and np.all(np.diff(wall[1:]) > 0), wall
    print(storage, [(round(w.chi_max, 4), "%.4e" % g[0], "%.4e" % g[1]) for w, g in zip(sweep, got)])
