"""Pins of the time integrators (Sec. 4) of the oracle."""
import json
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import brute, schemes, tensor
from paper_2510_21394_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example1_errors.json")


def _discrete_manufactured(ns, boxes, al, pars):
    """u(t) = (1+i) e^{-t} G exactly solves u' = K u + g(t, u) with the
    discrete source e^{-t}(1+i)(-G - K G - gamma G) + e^{-3t} 2 (kappa+i zeta)(1+i) G^3
    (K the dense matrix of O1), so only the time error remains."""
    nu, eta, gamma, kappa, zeta = pars
    P = tensor.Problem(ns, boxes, al, *pars)
    K = brute.kron_sum(P.As)
    X = P.mesh()
    G = np.exp(-sum(x ** 2 for x in X))
    KG = (K @ G.ravel()).reshape(P.shape)
    S1 = (1 + 1j) * (-G - KG - gamma * G)
    S3 = 2 * (kappa + 1j * zeta) * (1 + 1j) * G ** 3
    g = schemes.Nonlinearity(P, [-1.0, -3.0], [S1, S3])
    return P, g, (1 + 1j) * G, lambda t: (1 + 1j) * np.exp(-t) * G


ORDERS = [("lie", 1), ("lawson_euler", 1), ("etd2rk", 2), ("lawson_rk2", 2),
          ("krogstad", 4), ("lbdf2", 2)]


@pytest.mark.parametrize("scheme,order", ORDERS)
def test_time_order_on_discrete_manufactured_solution(scheme, order):
    P, g, u0, exact = _discrete_manufactured([10, 12], [(-3, 3), (-3.5, 3.5)], [1.3, 1.7],
                                             (1.0, 0.5, 1.0, 1.0, 0.5))
    S = tensor.Spectral(P)
    T = 0.5
    errs = []
    for m in (10, 20, 40):
        u = schemes.integrate(S, g, scheme, T / m, m, u0)
        errs.append(np.linalg.norm(u - exact(T)))
    rate = np.log2(errs[1] / errs[2])
    assert abs(rate - order) < 0.3, (scheme, errs, rate)


@pytest.mark.parametrize("scheme", ["lawson_euler", "lawson_rk2", "etd2rk", "krogstad", "strang"])
def test_exponential_schemes_exact_on_linear_problem(scheme):
    # gamma = kappa = zeta = 0 and no source: every exponential scheme reduces to exp(tau K) per step
    ns, boxes, al = [6, 7], [(-2, 2), (-2, 2)], [1.4, 1.6]
    P = tensor.Problem(ns, boxes, al, 1.0, 0.8, 0.0, 1.0, 0.0)
    P.kappa = 0.0
    S = tensor.Spectral(P)
    g = schemes.Nonlinearity(P)
    rng = np.random.default_rng(5)
    u0 = rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape)
    K = brute.kron_sum(P.As)
    T, m = 0.3, 7
    ref = brute.apply_exp(K, T, u0.ravel())
    if scheme == "strang":   # the exact flow needs kappa > 0; a tiny kappa with |u| ~ 1 stays linear to rounding
        P.kappa = 1e-300
    u = schemes.integrate(S, g, scheme, T / m, m, u0).ravel()
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_exact_nonlinear_flow_solves_its_ode():
    # phi_t(w) solves w' = gamma w - (kappa + i zeta)|w|^2 w  (Sec. 4, Strang splitting)
    P = tensor.Problem([3], [(-1, 1)], [1.5], 1.0, 0.0, 0.7, 1.3, -0.4)
    w0 = np.array([0.8 - 0.5j, 2.0 + 0.1j, 1e-3j])
    for t in (0.01, 0.4):
        got = schemes.exact_flow(P, t, w0)

        def rhs(_, y):
            w = y[:3] + 1j * y[3:]
            f = P.gamma * w - (P.kappa + 1j * P.zeta) * np.abs(w) ** 2 * w
            return np.concatenate([f.real, f.imag])
        sol = solve_ivp(rhs, (0, t), np.concatenate([w0.real, w0.imag]), rtol=1e-13, atol=1e-15, method="DOP853")
        ref = sol.y[:3, -1] + 1j * sol.y[3:, -1]
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-14)


def test_strang_second_order_self_convergence():
    P = tensor.Problem([9, 8], [(-4, 4), (-4, 4)], [1.3, 1.8], 1.0, 1.0, 1.0, 1.0, 1.0)
    S = tensor.Spectral(P)
    g = schemes.Nonlinearity(P)
    u0 = inputs.sech_pulse_noise([9, 8], [(-4, 4), (-4, 4)], amp=0.0)
    T = 0.5
    ref = schemes.integrate(S, g, "krogstad", T / 400, 400, u0)
    e = [np.linalg.norm(schemes.integrate(S, g, "strang", T / m, m, u0) - ref) for m in (10, 20, 40)]
    rate = np.log2(e[1] / e[2])
    assert abs(rate - 2) < 0.3


def _example1(order, scheme, m):
    n, al = 400, [1.2, 1.8]
    pars = dict(nu=1.0, eta=1.0, gamma=3.0, kappa=1.0, zeta=2.0)
    P = tensor.Problem([n, n], [(-1, 1)] * 2, al, *pars.values(), order=order)
    S = tensor.Spectral(P)
    u0, sig, Ss = inputs.polynomial_manufactured([n, n], al, **pars)
    g = schemes.Nonlinearity(P, sig, Ss)
    u = schemes.integrate(S, g, scheme, 1.0 / m, m, u0)
    return schemes.l2_error(P, u, inputs.polynomial_exact([n, n], 1.0))


def test_paper_example1_lbdf2_errors():
    gold = json.load(open(GOLDEN))["lbdf2_fd2"]
    for m, e in zip(gold["steps"], gold["errors"]):
        assert _example1(2, "lbdf2", m) == pytest.approx(e, rel=1e-4)


@pytest.mark.slow
def test_paper_example1_krogstad_fd4_errors():
    gold = json.load(open(GOLDEN))["krogstad_fd4"]
    for m, e in zip(gold["steps"], gold["errors"]):
        assert _example1(4, "krogstad", m) == pytest.approx(e, rel=1e-4)
