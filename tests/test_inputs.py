"""Pins of the closed-form continuous sources in the shared input module."""
import math

import mpmath
import numpy as np
import pytest

from paper_2510_21394_gb300 import inputs


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.8, 1.99])
def test_riesz_gaussian_against_mpmath(alpha):
    mpmath.mp.dps = 30
    xs = np.linspace(0, 20, 161)
    got = inputs.riesz_gaussian(xs, alpha)
    a = (1 + alpha) / 2
    ref = np.array([float(-(2 ** alpha) * mpmath.gamma(a) / mpmath.sqrt(mpmath.pi)
                          * mpmath.hyp1f1(a, 0.5, -mpmath.mpf(x) ** 2)) for x in xs])
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def test_riesz_gaussian_fourier_definition():
    # -1/pi int_0^inf xi^alpha sqrt(pi) e^{-xi^2/4} cos(xi x) d xi (Fourier symbol -|xi|^alpha)
    mpmath.mp.dps = 25
    for alpha in (1.3, 1.7):
        for x in (0.0, 0.8, 2.1):
            f = lambda s: s ** alpha * mpmath.sqrt(mpmath.pi) * mpmath.exp(-s * s / 4) * mpmath.cos(s * x)
            ref = -float(mpmath.quad(f, [0, mpmath.inf])) / math.pi
            assert inputs.riesz_gaussian(np.array([x]), alpha)[0] == pytest.approx(ref, rel=1e-10, abs=1e-14)


def test_riesz_gaussian_alpha_two_limit():
    x = np.linspace(-3, 3, 13)
    np.testing.assert_allclose(inputs.riesz_gaussian(x, 1.9999999), (4 * x ** 2 - 2) * np.exp(-x ** 2), atol=3e-6)


def test_riesz_poly_alpha_two_limit():
    x = np.linspace(-0.95, 0.95, 11)
    d2 = -8 * (1 - x ** 2) ** 3 + 48 * x ** 2 * (1 - x ** 2) ** 2
    np.testing.assert_allclose(inputs.riesz_poly(x, 1.9999999), d2, atol=2e-5)


def test_riesz_poly_against_integral_definition():
    # left RL derivative by the defining integral, differentiated twice by mpmath
    mpmath.mp.dps = 30
    alpha = 1.4
    w = lambda s: (1 - s * s) ** 4

    def left(x):
        I = lambda y: mpmath.quad(lambda s: (y - s) ** (1 - alpha) * w(s), [-1, y])
        return mpmath.diff(I, x, 2) / mpmath.gamma(2 - alpha)

    def right(x):
        I = lambda y: mpmath.quad(lambda s: (s - y) ** (1 - alpha) * w(s), [y, 1])
        return mpmath.diff(I, x, 2) / mpmath.gamma(2 - alpha)
    for x in (-0.3, 0.45):
        ref = -float(left(x) + right(x)) / (2 * math.cos(alpha * math.pi / 2))
        assert inputs.riesz_poly(np.array([x]), alpha)[0] == pytest.approx(ref, rel=1e-8)


def test_seeded_inputs_are_deterministic():
    a = inputs.gaussian_random_phase([12, 10, 8], [(-10, 10)] * 3, seed=1)
    b = inputs.gaussian_random_phase([12, 10, 8], [(-10, 10)] * 3, seed=1)
    assert a.shape == (8, 10, 12) and np.array_equal(a, b)
    np.testing.assert_allclose(np.abs(a), np.abs(inputs.gaussian_pulse([12, 10, 8], [(-10, 10)] * 3)), rtol=1e-14)
    c = inputs.sech_pulse_noise([6, 5], [(-20, 20)] * 2, seed=0)
    assert c.shape == (5, 6) and c.dtype == np.complex128


def test_batched_instances_ranges_and_determinism():
    a = inputs.batched_instances()
    b = inputs.batched_instances()
    assert a == b and len(a) == 96
    two = [s for s in a if len(s["ns"]) == 2]
    three = [s for s in a if len(s["ns"]) == 3]
    assert len(two) == 64 and len(three) == 32
    assert all(128 <= s["ns"][0] <= 768 and s["ns"][0] == s["ns"][1] for s in two)
    assert all(48 <= s["ns"][0] <= 160 and len(set(s["ns"])) == 1 for s in three)
    for s in a:
        assert all(1.1 <= al <= 1.9 for al in s["alphas"]) and len(s["alphas"]) == len(s["ns"])
        assert 0.5 <= s["nu"] <= 2 and -1 <= s["eta"] <= 1 and -1 <= s["zeta"] <= 1
        assert 0 <= s["gamma"] <= 1 and 0.5 <= s["kappa"] <= 2
        assert s["boxes"] == [(-10.0, 10.0)] * len(s["ns"])
