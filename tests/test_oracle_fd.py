"""Pins of the finite-difference part of the oracle (paper Sec. 2)."""
import mpmath
import numpy as np
import pytest

from oracle import fd
from paper_2510_21394_gb300 import inputs


@pytest.mark.parametrize("alpha", [1.1, 1.35, 1.5, 1.8, 1.95])
def test_recurrence_matches_direct_gamma_formula(alpha):
    # g_k = (-1)^k Gamma(alpha+1) / (Gamma(alpha/2-k+1) Gamma(alpha/2+k+1)), Sec. 2
    mpmath.mp.dps = 40
    g = fd.g_coeffs(alpha, 60)
    for k in range(60):
        a = mpmath.mpf(alpha)
        ref = (-1) ** k * mpmath.gamma(a + 1) / (mpmath.gamma(a / 2 - k + 1) * mpmath.gamma(a / 2 + k + 1))
        assert abs(g[k] - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300


def test_alpha_two_is_second_difference():
    g = fd.g_coeffs(2.0, 8)
    np.testing.assert_allclose(g, [2, -1, 0, 0, 0, 0, 0, 0], atol=1e-15)


def test_fd4_alpha_two_is_pentadiagonal():
    g = fd.g_coeffs_fd4(2.0, 8)
    np.testing.assert_allclose(g, [5 / 2, -4 / 3, 1 / 12, 0, 0, 0, 0, 0], atol=1e-15)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_D_symmetric_toeplitz_negative_definite(alpha, order):
    n, h = 37, 0.13
    D = fd.D_matrix(n, alpha, h, order)
    assert np.array_equal(D, D.T)
    for k in range(n):
        assert np.all(np.diag(D, k) == D[0, k])
    w = np.linalg.eigvalsh(D)
    assert w.max() < 0
    if order == 2:   # Gershgorin: sum_{k>=1}|g_k| < g_0/2 so lam in [-2 g_0 h^-alpha, 0)
        g0 = fd.g_coeffs(alpha, 1)[0]
        assert w.min() >= -2 * g0 * h ** (-alpha) * (1 + 1e-14)


@pytest.mark.parametrize("alpha", [1.3, 1.7])
def test_coefficients_sum_to_zero(alpha):
    g = fd.g_coeffs(alpha, 200000)
    assert abs(g[0] + 2 * g[1:].sum()) < 1e-5


@pytest.mark.parametrize("alpha", [1.2, 1.8])
def test_fd_orders_against_continuous_riesz(alpha):
    # D_n^alpha w -> Riesz derivative of w = (1-x^2)^4 on (-1,1): O(h^2) (Eq. FD2), faster for Eq. FD4
    errs = {2: [], 4: []}
    for n in (99, 199, 399):
        x, h = fd.grid(n, -1.0, 1.0)
        w = (1 - x ** 2) ** 4
        ex = inputs.riesz_poly(x, alpha)
        for order in (2, 4):
            errs[order].append(np.sqrt(h * np.sum((fd.D_matrix(n, alpha, h, order) @ w - ex) ** 2)))
    r2 = np.log2(errs[2][1] / errs[2][2])
    r4 = np.log2(errs[4][1] / errs[4][2])
    assert 1.8 < r2 < 2.3
    # (1-x^2)^4 has a jump in its 4th derivative at +-1, which caps the FD4 rate
    assert r4 > 2.5 and errs[4][2] < errs[2][2] / 50
