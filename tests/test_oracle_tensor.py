"""Pins of O2 (tensor form, Sec. 3.2) against O1 and against definitions."""
import itertools

import numpy as np
import pytest

from oracle import brute, tensor

CASES = [
    ([7, 9], [(-1.0, 1.0), (-3.0, 2.0)], [1.2, 1.8]),
    ([5, 6, 8], [(-2.0, 2.0), (-1.0, 3.0), (-1.5, 1.5)], [1.2, 1.8, 1.5]),
    ([11], [(-1.0, 1.0)], [1.4]),
]


def _prob(ns, boxes, al, order=2):
    return tensor.Problem(ns, boxes, al, 1.0, 0.6, 0.5, 1.0, -0.3, order=order)


def test_mode_product_against_loops():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(3, 4, 5)) + 1j * rng.normal(size=(3, 4, 5))   # (n3, n2, n1)
    Ms = {1: rng.normal(size=(5, 5)), 2: rng.normal(size=(4, 4)), 3: rng.normal(size=(3, 3))}
    for mu, M in Ms.items():
        Y = tensor.mode_product(X, M, mu)
        Yr = np.zeros_like(X)
        for j3, j2, j1 in itertools.product(range(3), range(4), range(5)):
            j = [j1, j2, j3]
            s = 0
            for k in range(M.shape[0]):
                jk = list(j)
                jk[mu - 1] = k
                s += M[j[mu - 1], k] * X[jk[2], jk[1], jk[0]]
            Yr[j3, j2, j1] = s
        np.testing.assert_allclose(Y, Yr, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("ns,boxes,al", CASES)
def test_eig_residuals(ns, boxes, al):
    P = _prob(ns, boxes, al)
    S = tensor.Spectral(P)
    for D, Q, w in zip(P.Ds, S.Q, S.lam):
        assert np.linalg.norm(D @ Q - Q * w) <= 1e-13 * np.linalg.norm(D)
        assert np.linalg.norm(Q.T @ Q - np.eye(len(w))) <= 1e-13


@pytest.mark.parametrize("ns,boxes,al", CASES)
def test_K_apply_equals_dense_K(ns, boxes, al):
    P = _prob(ns, boxes, al)
    K = brute.kron_sum(P.As)
    rng = np.random.default_rng(1)
    U = rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape)
    np.testing.assert_allclose(tensor.K_apply(P, U).ravel(), K @ U.ravel(), rtol=1e-12, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("ns,boxes,al", CASES)
@pytest.mark.parametrize("order", [2, 4])
def test_apply_f_against_brute_force(ns, boxes, al, order):
    P = _prob(ns, boxes, al, order)
    S = tensor.Spectral(P)
    K = brute.kron_sum(P.As)
    rng = np.random.default_rng(2)
    V = rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape)
    v = V.ravel()
    for th in (1e-3, 0.05):
        cases = [("inv", 0, brute.apply_inv(K, th, v)), ("exp", 0, brute.apply_exp(K, th, v))]
        phis = brute.apply_phis(K, th, v, 3)
        cases += [("phi", l + 1, phis[l]) for l in range(3)]
        for kind, ell, ref in cases:
            got = S.apply_f(kind, ell, th, V).ravel()
            assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), (kind, ell, th)
        got = S.apply_exp_kron(th, V).ravel()
        assert np.linalg.norm(got - cases[1][2]) <= 1e-13 * np.linalg.norm(cases[1][2])


def test_phi_zero_order_is_exp():
    P = _prob(*CASES[0])
    S = tensor.Spectral(P)
    V = np.ones(P.shape, dtype=complex)
    np.testing.assert_allclose(S.apply_f("phi", 0, 0.1, V), S.apply_f("exp", 0, 0.1, V), rtol=1e-14)
