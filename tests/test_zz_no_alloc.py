"""The allocation-free diagnostics entry point, for callers that cannot let a
library allocate device memory (a host application with its own fixed device
memory pool, or a latency-critical loop that cannot afford cudaMalloc).

It is checked through the C ABI against the handle-based lbm_diagnostics on
the same state, within the diagnostics tolerance of the parity tests, on two
calls in a row (the second call reuses the static scratch the first one left
behind).  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

REL = {"f64": 1e-12, "f32": 1e-6, "f16dev": 1e-6, "bf16dev": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _close(got, want, rel):
    scale = np.abs(want) + np.abs(want[:1]) * 1e-3 + 1e-300
    assert np.all(np.abs(got - want) <= rel * scale), (got, want)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16dev", "bf16dev"])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_noalloc_diagnostics_match_lbm_diagnostics(storage, bc):
    """Every storage format (the 16-bit ones decode with their per-plane scales)
    and both accepted boundaries (the periodic pull wraps)."""
    import torch

    from paper_1203_6350_gb300 import lbm

    w = wl.small_pulse("II", storage).with_(u0=(0.05, 0.0), u_f=(0.05, 0.0), bc=bc)
    lat = lbm.Lattice.from_workload(w)
    lat.step(80)
    state = torch.empty(lat.state_bytes(), dtype=torch.uint8, device="cuda")
    rc, t = lbm.lbm_get_state(lat.h, state.data_ptr(), state.numel(), 1)
    assert rc == 0 and t == 80
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for region in [(0, 0, w.nx, w.ny), (20, 20, 80, 80), (3, 0, 4, 100), (7, 7, 7, 7)]:
        want = lat.diagnostics(region)
        for _ in range(2):  # two calls in a row
            out = np.full(6, np.nan)
            rc = lbm.lbm_diagnostics_noalloc(
                state.data_ptr(), lbm.STORAGE[storage], w.nx, w.ny, lbm.BC[w.bc], w.rho0,
                w.u0[0], w.u0[1], *region, out.ctypes.data, 0, stream)
            assert rc == lbm.LBM_OK
            _close(out, want, REL[storage])
        dev = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lbm.lbm_diagnostics_noalloc(
            state.data_ptr(), lbm.STORAGE[storage], w.nx, w.ny, lbm.BC[w.bc], w.rho0, w.u0[0],
            w.u0[1], *region, dev.data_ptr(), 1, stream)
        assert rc == lbm.LBM_OK
        torch.cuda.synchronize()
        _close(dev.cpu().numpy(), want, REL[storage])
    lat.close()


def test_noalloc_rejects_inputs_beyond_the_static_scratch():
    from paper_1203_6350_gb300 import lbm

    out = np.zeros(6)
    # 20000 x 20000 = 4e8 cells > 268,435,456: rejected before any device work
    rc = lbm.lbm_diagnostics_noalloc(1, lbm.STORAGE["f32"], 20000, 20000, 0, 1.0, 0.0, 0.0,
                                     0, 0, 20000, 20000, out.ctypes.data, 0, None)
    assert rc == lbm.LBM_ERR_TOO_LARGE
    rc = lbm.lbm_diagnostics_noalloc(None, lbm.STORAGE["f32"], 16, 16, 0, 1.0, 0.0, 0.0,
                                     0, 0, 16, 16, out.ctypes.data, 0, None)
    assert rc == lbm.LBM_ERR_ARG
