"""Pins of O1 (dense Kronecker sum, dense solve/expm/augmented expm)."""
import itertools
import math

import mpmath
import numpy as np
import pytest

from oracle import brute
from oracle.phi import phi

NS3 = [5, 6, 8]
AL3 = [1.2, 1.8, 1.5]
BOX3 = [(-2.0, 2.0), (-1.0, 3.0), (-1.5, 1.5)]


def test_kron_sum_against_index_definition():
    # K[j, j'] = sum_mu A_mu[j_mu, j'_mu] prod_{nu != mu} delta(j_nu, j'_nu),
    # with j = j_1 + n_1 (j_2 - 1) + n_1 n_2 (j_3 - 1) (Eq. indexj, Eq. Ksum)
    rng = np.random.default_rng(0)
    ns = [3, 4, 2]
    As = [rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) for n in ns]
    K = brute.kron_sum(As)
    N = int(np.prod(ns))
    Kref = np.zeros((N, N), dtype=complex)
    idx = lambda j: j[0] + ns[0] * j[1] + ns[0] * ns[1] * j[2]
    for j in itertools.product(*[range(n) for n in ns]):
        for jp in itertools.product(*[range(n) for n in ns]):
            v = 0
            for mu in range(3):
                if all(j[o] == jp[o] for o in range(3) if o != mu):
                    v += As[mu][j[mu], jp[mu]]
            Kref[idx(j), idx(jp)] = v
    np.testing.assert_array_equal(K, Kref)


def test_expm_two_ways():
    K = brute.K_matrix([4, 5], [1.3, 1.7], [(-1, 1), (-2, 2)], 1.0, 0.7)
    for th in (1e-3, 0.05):
        from scipy.linalg import expm
        A = expm(th * K)
        B = brute.expm_taylor(th * K)
        assert np.linalg.norm(A - B) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_augmented_phi_scalar_case(ell):
    # N = 1: phi_ell(theta K) v is the scalar phi_ell(theta k) v
    mpmath.mp.dps = 150
    for k in (-3.0 + 1.0j, -0.2, 5e-5 - 1e-5j):
        K = np.array([[k]], dtype=complex)
        got = brute.apply_phi(K, 0.7, np.array([2.0 - 1.0j]), ell)[0]
        z = mpmath.mpc(0.7 * k)
        p = mpmath.exp(z)
        for l in range(1, ell + 1):
            p = (p - mpmath.mpf(1) / mpmath.factorial(l - 1)) / z
        ref = complex(p) * (2.0 - 1.0j)
        assert abs(got - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_augmented_phi_zero_matrix(ell):
    K = np.zeros((6, 6), dtype=complex)
    v = np.arange(6) + 1j
    np.testing.assert_allclose(brute.apply_phi(K, 1.0, v, ell), v / math.factorial(ell), rtol=1e-15)


def test_augmented_phi_recurrence_on_matrices():
    # phi_l(A) v = A phi_{l+1}(A) v + v / l!  (Eq. phi applied to a matrix argument)
    K = brute.K_matrix([4, 3], [1.4, 1.6], [(-1, 1), (-1, 1)], 1.0, -0.5)
    rng = np.random.default_rng(1)
    v = rng.normal(size=12) + 1j * rng.normal(size=12)
    th = 0.02
    phis = brute.apply_phis(K, th, v, 4)
    allp = [brute.apply_exp(K, th, v)] + phis
    for l in range(4):
        lhs = allp[l]
        rhs = th * K @ allp[l + 1] + v / math.factorial(l)
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)


def test_inverse_solves_sylvester_2d():
    # f(z) = 1/(1-z): (I1/2 - th A1) X + X (I2/2 - th A2)^T = V  (Sec. 3.1)
    ns, al, box = [7, 9], [1.2, 1.8], [(-1, 1), (-3, 3)]
    Ds = brute.assemble_D(ns, al, box)
    c = 1.0 + 0.5j
    As = [c * D for D in Ds]
    K = brute.kron_sum(As)
    rng = np.random.default_rng(2)
    V = rng.normal(size=(9, 7)) + 1j * rng.normal(size=(9, 7))   # shape (n2, n1): V.ravel() is vec
    th = 0.03
    x = brute.apply_inv(K, th, V.ravel())
    X = x.reshape(9, 7).T            # X[j1, j2]
    Vm = V.T
    R = (np.eye(7) / 2 - th * As[0]) @ X + X @ (np.eye(9) / 2 - th * As[1]).T - Vm
    assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(Vm)


def test_exp_kron_is_product_of_small_exponentials():
    # exp(theta K) = exp(theta A_2) x exp(theta A_1)  (Sec. 3.1, commuting Kronecker terms)
    from scipy.linalg import expm
    ns, al, box = [4, 5], [1.5, 1.3], [(-1, 1), (-2, 2)]
    Ds = brute.assemble_D(ns, al, box)
    As = [(1.0 + 1.0j) * D for D in Ds]
    K = brute.kron_sum(As)
    th = 0.01
    A = expm(th * K)
    B = np.kron(expm(th * As[1]), expm(th * As[0]))
    assert np.linalg.norm(A - B) <= 1e-13 * np.linalg.norm(A)
