"""Input recipes: the sponge profiles of Table tab:sigma, pinned by their
closed forms (the polynomial profile's integral is its strength A; with
power 4 it is the normalised profile of Eq. (normalizedsigma))."""
import numpy as np
import pytest

import workloads as wl


@pytest.mark.parametrize("power", [2, 3, 4, 6])
def test_polynomial_profile_integrates_to_its_strength(power):
    """Unit spacing on a profile that vanishes at both ends is the trapezoid
    rule: the sum over one layer's cells tends to A as O(1 / width^2)."""
    for width, tol in ((50, 2e-3), (400, 4e-5)):
        chi = wl.polynomial_profile(3 * width, width, A=2.5, power=power)
        one_layer = chi[:width]  # the left layer, depths width .. 1
        assert abs(one_layer.sum() - 2.5) <= tol * 2.5
        assert np.all(chi[width:2 * width] == 0.0)  # the interior is undamped


def test_polynomial_profile_power_four_is_the_normalised_profile():
    """Eq. (normalizedsigma): chi 3125 / (256 (L - x0)^5) = A (n + 1)(n + 2) /
    (L - x0)^(n + 2) for n = 4, i.e. A = chi (L - x0) 3125 / (256 * 30)."""
    chi = 0.7
    a = wl.polynomial_profile(300, 64, A=chi * 65 * 3125 / (256 * 30), power=4)
    b = wl.orszag_profile(300, 64, chi)
    np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)


def test_polynomial_profile_peaks_at_n_over_n_plus_one():
    """d/dt t^n (1 - t) = 0 at t = n / (n + 1): 80 % into the layer for n = 4."""
    width = 99  # L = 100: depth 80 is the peak for n = 4, 75 for n = 3
    for power, peak in ((4, 80), (3, 75)):
        chi = wl.polynomial_profile(3 * width, width, A=1.0, power=power)
        d = wl.layer_depth(3 * width, width)
        assert d[np.argmax(chi)] == peak
