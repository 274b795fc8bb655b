"""Pins of the oracle's discrete adjoint (Lawson-RK2) against finite differences
and dot-product identities (gradients in the sense dJ/dRe + i dJ/dIm)."""
import numpy as np
import pytest

from oracle import adjoint, schemes, tensor
from paper_2510_21394_gb300 import inputs

NS = [9, 7, 6]
BOXES = [(-3.0, 3.0), (-2.5, 2.5), (-2.0, 2.0)]
AL = [1.5, 1.3, 1.7]
PARS = [1.0, 0.5, 0.8, 1.2, 0.4]     # nu, eta, gamma, kappa, zeta


def _setup(pars, with_source=True):
    P = tensor.Problem(NS, BOXES, AL, *pars)
    S = tensor.Spectral(P)
    rng = np.random.default_rng(11)
    src = [0.2 * (rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape))] if with_source else []
    g = schemes.Nonlinearity(P, [-0.5 + 1.0j] if with_source else [], src)
    return P, S, g


def _u0():
    u = inputs.gaussian_pulse(NS, [(-2.0, 2.0)] * 3)
    rng = np.random.default_rng(3)
    return u * np.exp(1j * rng.uniform(0, 1, size=u.shape))


def test_dot_product_identities():
    P, S, _ = _setup(PARS)
    rng = np.random.default_rng(0)
    x, y, u = (rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape) for _ in range(3))
    # g linearisation
    lhs = np.real(np.vdot(adjoint.g_linear(P, u, x), y))
    rhs = np.real(np.vdot(x, adjoint.g_adjoint(P, u, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # exp(tau K) and its adjoint
    lhs = np.real(np.vdot(S.apply_exp_kron(0.01, x), y))
    rhs = np.real(np.vdot(x, adjoint.exp_h(S, 0.01, y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_lawson_rk2_forward_matches_scheme():
    P, S, g = _setup(PARS)
    u0 = _u0()
    us, _ = adjoint.forward(S, g, 0.02, 5, u0)
    ref = schemes.integrate(S, g, "lawson_rk2", 0.02, 5, u0)
    np.testing.assert_allclose(us[-1], ref, rtol=0, atol=1e-14)


def test_gradient_against_central_differences():
    tau, m = 0.02, 6
    P, S, g = _setup(PARS)
    u0 = _u0()
    target = 0.9 * adjoint.forward(S, g, tau, m, u0)[0][-1] + 0.01
    J, gu, gp = adjoint.gradient(S, g, tau, m, u0, target)
    # u0: directional derivative along a random complex direction
    rng = np.random.default_rng(7)
    d = rng.normal(size=u0.shape) + 1j * rng.normal(size=u0.shape)
    eps = 1e-6
    fd = (adjoint.loss(S, g, tau, m, u0 + eps * d, target) - adjoint.loss(S, g, tau, m, u0 - eps * d, target)) / (2 * eps)
    assert np.real(np.vdot(gu, d)) == pytest.approx(fd, rel=1e-6)
    # parameters
    for k in range(5):
        pp, pm = list(PARS), list(PARS)
        h = 1e-6 * max(1.0, abs(PARS[k]))
        pp[k] += h
        pm[k] -= h
        Pp, Sp, gpp = _setup(pp)
        Pm, Sm, gpm = _setup(pm)
        fd = (adjoint.loss(Sp, gpp, tau, m, u0, target) - adjoint.loss(Sm, gpm, tau, m, u0, target)) / (2 * h)
        assert gp[k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(J)), (k, gp[k], fd)
