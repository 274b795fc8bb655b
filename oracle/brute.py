"""O1: brute-force f(theta K) v with the dense Kronecker sum (tiny grids only).

No eigendecomposition is used anywhere in this module:

* K is assembled densely as in Eq. Ksum,
  K = sum_mu I_d x ... x I_{mu+1} x A_mu x I_{mu-1} x ... x I_1,
  A_mu = (nu + i eta) D_mu, so that the vec index has j_1 fastest (Eq. indexj).
* (1 - z)^{-1}: dense LU solve of (I - theta K) x = v.
* e^z: scipy's Pade scaling-and-squaring ``expm``.
* phi_l: the top-right block of the exponential of the augmented matrix
  [[theta K, v e_1^T], [0, J_l]], J_l the l x l upper shift; its columns are
  phi_1(theta K) v, ..., phi_l(theta K) v (exponential of a block-triangular
  matrix; Saad 1992, Al-Mohy & Higham 2011 Thm 2.1).  No division by z.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np
import scipy.linalg as sla

from . import fd


def assemble_D(ns, alphas, boxes, order=2):
    """Per-direction D_mu (Eq. Dnalpha) on the interior grids of Sec. 2."""
    Ds = []
    for n, al, (a, b) in zip(ns, alphas, boxes):
        _, h = fd.grid(n, a, b)
        Ds.append(fd.D_matrix(n, al, h, order))
    return Ds


def kron_sum(As):
    """K = A_d (+) ... (+) A_1 (Eq. Ksum); As = [A_1, ..., A_d]."""
    ns = [A.shape[0] for A in As]
    d = len(As)
    N = int(np.prod(ns))
    K = np.zeros((N, N), dtype=np.complex128)
    for mu in range(d):
        term = np.ones((1, 1), dtype=np.complex128)
        for nu in reversed(range(d)):          # factors from direction d down to 1
            term = np.kron(term, As[mu] if nu == mu else np.eye(ns[nu]))
        K += term
    return K


def K_matrix(ns, alphas, boxes, nu, eta, order=2):
    Ds = assemble_D(ns, alphas, boxes, order)
    return kron_sum([(nu + 1j * eta) * D for D in Ds])


def apply_inv(K, theta, v):
    """(I - theta K)^{-1} v by a dense solve."""
    N = K.shape[0]
    return np.linalg.solve(np.eye(N) - theta * K, v)


def apply_exp(K, theta, v):
    return sla.expm(theta * K) @ v


def apply_phis(K, theta, v, ell):
    """[phi_1(theta K) v, ..., phi_ell(theta K) v] from one augmented expm."""
    N = K.shape[0]
    Aug = np.zeros((N + ell, N + ell), dtype=np.complex128)
    Aug[:N, :N] = theta * K
    Aug[:N, N] = v
    for i in range(ell - 1):
        Aug[N + i, N + i + 1] = 1.0
    E = sla.expm(Aug)
    return [E[:N, N + l] for l in range(ell)]


def apply_phi(K, theta, v, ell):
    if ell == 0:
        return apply_exp(K, theta, v)
    return apply_phis(K, theta, v, ell)[ell - 1]


def expm_taylor(M, tol=1e-18):
    """Independent check of scipy.expm: Taylor series with scaling and
    squaring (e^M = (e^{M/2^s})^{2^s})."""
    nrm = np.linalg.norm(M, 1)
    s = max(0, int(np.ceil(np.log2(max(nrm, 1e-300)))) + 1)
    A = M / 2.0 ** s
    E = np.eye(M.shape[0], dtype=np.complex128)
    T = E.copy()
    for k in range(1, 60):
        T = T @ A / k
        E = E + T
        if np.linalg.norm(T, 1) < tol * np.linalg.norm(E, 1):
            break
    for _ in range(s):
        E = E @ E
    return E
