"""The bandwidth probe behind the benchmark's L2 roofline denominator
(lbm_probe_copy): it must really copy -- after an odd number of passes b holds
a's data, after an even number a is unchanged -- on sizes that leave ragged
last strides, and it refuses bad arguments before any device work."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("words", [1, 1000, 311_296 + 17, 2_359_296])
def test_probe_copies(words):
    import torch

    from paper_1203_6350_gb300 import lbm

    n = 4 * words  # float32 elements, 16 bytes per word
    a = torch.arange(n, dtype=torch.float32, device="cuda")
    ref = a.clone()
    for iters in (1, 2, 5):
        b = torch.full_like(a, -1.0)
        assert lbm.lbm_probe_copy(a.data_ptr(), b.data_ptr(), 16 * words, iters, None) == lbm.LBM_OK
        torch.cuda.synchronize()
        assert torch.equal(b, ref)  # the first pass wrote b, later passes copy it back and forth
        assert torch.equal(a, ref)


def test_probe_rejects_bad_arguments():
    import torch

    from paper_1203_6350_gb300 import lbm

    a = torch.zeros(64, dtype=torch.float32, device="cuda")
    b = torch.zeros(64, dtype=torch.float32, device="cuda")
    p, q = a.data_ptr(), b.data_ptr()
    assert lbm.lbm_probe_copy(None, q, 256, 1, None) == lbm.LBM_ERR_ARG
    assert lbm.lbm_probe_copy(p, q, 250, 1, None) == lbm.LBM_ERR_ARG   # not a multiple of 16
    assert lbm.lbm_probe_copy(p, q, 256, 0, None) == lbm.LBM_ERR_ARG   # no pass
    assert lbm.lbm_probe_copy(p + 4, q, 240, 1, None) == lbm.LBM_ERR_ARG  # unaligned
