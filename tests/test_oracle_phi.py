"""Pins of the scalar phi-functions (Eq. phi)."""
import math

import mpmath
import numpy as np
import pytest

from oracle.phi import phi

ZS = [0.0, 1e-12, -3e-8 + 1e-8j, 1e-4, -2.5e-4 + 1e-4j, 0.3 - 0.2j, -0.99, 0.999j,
      -1.001, 1.5 + 1j, -2.4 - 1.2j, -7.0, 3.0 + 4.0j, -60.0 + 30.0j, -600.0 - 300.0j]


def _phi_mp(ell, z):
    mpmath.mp.dps = 150
    z = mpmath.mpc(z)
    if z == 0:
        return mpmath.mpf(1) / mpmath.factorial(ell)
    p = mpmath.exp(z)
    for l in range(1, ell + 1):
        p = (p - mpmath.mpf(1) / mpmath.factorial(l - 1)) / z
    return complex(p)


@pytest.mark.parametrize("ell", [0, 1, 2, 3, 4])
def test_phi_against_mpmath(ell):
    for z in ZS:
        ref = _phi_mp(ell, z)
        got = complex(phi(ell, z))
        assert abs(got - ref) <= 4e-15 * abs(ref), (ell, z, got, ref)


def test_phi_at_zero():
    for ell in range(6):
        assert phi(ell, 0.0) == pytest.approx(1.0 / math.factorial(ell), rel=1e-16)


def test_phi_recurrence_identity():
    rng = np.random.default_rng(3)
    z = rng.normal(size=200) * 3 + 1j * rng.normal(size=200) * 3
    z = np.concatenate([z, 1e-3 * z])
    for ell in range(4):
        lhs = phi(ell, z)
        rhs = z * phi(ell + 1, z) + 1.0 / math.factorial(ell)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-15)
