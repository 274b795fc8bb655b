"""O2: tensor-form f(theta K) v in FP64 (paper Sec. 3).

Tensors are numpy arrays of shape (n_d, ..., n_1) in C order, so that
``U.ravel()`` is vec(U) with j_1 fastest (Eq. indexj).  Direction mu lives on
axis d - mu.

* ``mode_product(X, M, mu)``: X x_mu M, i.e. M multiplied onto every
  mu-fiber (Sec. 3.2), as a BLAS matmul on a moved axis.
* ``Spectral``: per-direction eigendecompositions D_mu = Q_mu Lam_mu Q_mu^T
  (Eq. diag, numpy ``eigh``), the eigenvalues of K as the direct sum
  (nu + i eta) sum_mu lam_{j_mu} (Sec. 3.2) and
  f(theta K) v = ((F o (V x_1 Q_1^T ... x_d Q_d^T)) x_1 Q_1 ... x_d Q_d)
  (Eq. fKu_diag), with the exponential also in the Kronecker-product form
  V x_1 exp(theta A_1) ... x_d exp(theta A_d) (Eq. Neudeckerd).
* ``K_apply``: K u = vec(sum_mu U x_mu A_mu) (Eq. kronsumv), no eig.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

from . import fd
from .phi import phi


def mode_product(X, M, mu):
    """Y = X x_mu M:  Y[.., i, ..] = sum_k M[i, k] X[.., k, ..] on direction mu."""
    ax = X.ndim - mu
    Xm = np.moveaxis(X, ax, -1)
    Y = Xm @ M.T
    return np.moveaxis(Y, -1, ax)


def tucker(X, Ms):
    """X x_1 M_1 x_2 ... x_d M_d."""
    for mu, M in enumerate(Ms, start=1):
        X = mode_product(X, M, mu)
    return X


def scalar_f(kind, ell, z):
    """f(z) for kind in {'inv': 1/(1-z), 'exp': e^z, 'phi': phi_ell(z)}."""
    if kind == "inv":
        return 1.0 / (1.0 - z)
    if kind == "exp":
        return np.exp(z)
    if kind == "phi":
        return phi(ell, z)
    raise ValueError(kind)


class Problem:
    """Parameters of the semidiscrete FCGLE (Sec. 2): grid, D_mu, nu..zeta."""

    def __init__(self, ns, boxes, alphas, nu, eta, gamma, kappa, zeta, order=2):
        self.d = len(ns)
        self.ns = list(ns)
        self.boxes = [tuple(b) for b in boxes]
        self.alphas = list(alphas)
        self.nu, self.eta = float(nu), float(eta)
        self.gamma, self.kappa, self.zeta = float(gamma), float(kappa), float(zeta)
        self.order = order
        self.xs, self.hs, self.Ds = [], [], []
        for n, (a, b), al in zip(ns, boxes, alphas):
            x, h = fd.grid(n, a, b)
            self.xs.append(x)
            self.hs.append(h)
            self.Ds.append(fd.D_matrix(n, al, h, order))
        self.c = self.nu + 1j * self.eta
        self.As = [self.c * D for D in self.Ds]
        self.shape = tuple(reversed(self.ns))        # (n_d, ..., n_1)
        self.N = int(np.prod(self.ns))

    def mesh(self):
        """Coordinate arrays x_mu broadcast to shape (n_d, ..., n_1)."""
        return np.meshgrid(*reversed(self.xs), indexing="ij")[::-1]

    def cell(self):
        return float(np.prod(self.hs))


def K_apply(P, U):
    """K u = vec(sum_mu U x_mu A_mu)  (Eq. kronsumv)."""
    out = np.zeros_like(U, dtype=np.complex128)
    for mu, A in enumerate(P.As, start=1):
        out += mode_product(U, A, mu)
    return out


class Spectral:
    """Eigen-data of K = Q Lam Q^T (Sec. 3.1-3.2) from numpy eigh."""

    def __init__(self, P):
        self.P = P
        self.Q, self.lam = [], []
        for D in P.Ds:
            w, V = np.linalg.eigh(D)
            self.Q.append(V)
            self.lam.append(w)
        # lam_{j_1..j_d} = (nu + i eta) sum_mu lam_{j_mu}, shape (n_d..n_1)
        L = np.zeros(P.shape)
        for mu, w in enumerate(self.lam, start=1):
            shp = [1] * P.d
            shp[P.d - mu] = len(w)
            L = L + w.reshape(shp)
        self.Lam = P.c * L
        self._F = {}

    def fwd(self, V):
        return tucker(V, [Q.T for Q in self.Q])

    def bwd(self, W):
        return tucker(W, self.Q)

    def F(self, kind, ell, theta):
        """F = f(theta lam_{j_1..j_d}); computed once per (f, theta) like the
        paper's R_theta and P_{l,theta} tensors (Sec. 4.1)."""
        key = (kind, ell if kind == "phi" else 0, float(theta))
        if key not in self._F:
            self._F[key] = scalar_f(kind, ell, theta * self.Lam)
        return self._F[key]

    def apply_f(self, kind, ell, theta, V):
        """f(theta K) v in the Tucker form (Eq. fKu_diag)."""
        return self.bwd(self.F(kind, ell, theta) * self.fwd(V))

    def E(self, theta):
        """E_mu = exp(theta A_mu) = Q_mu diag(e^{theta (nu+i eta) lam_mu}) Q_mu^T."""
        return [(Q * np.exp(theta * self.P.c * w)) @ Q.T for Q, w in zip(self.Q, self.lam)]

    def apply_exp_kron(self, theta, V):
        """exp(theta K) v = V x_1 E_1 ... x_d E_d  (Eq. Neudeckerd)."""
        return tucker(V, self.E(theta))
