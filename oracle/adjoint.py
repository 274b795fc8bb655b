"""Discrete adjoint of the Heun-based Lawson-RK2 scheme, FP64 (oracle).

Forward step (the reading in ``schemes.lawson_rk2_step``), E = exp(tau K):
    k1 = g(t, u);  a = u + tau k1;  v = E a;  b = u + tau/2 k1;  w = E b;
    u' = w + tau/2 g(t + tau, v).
Misfit J = 1/2 sum_j |u_j(T) - u_target,j|^2 (no cell volume); gradients are
taken in the real sense, grad_u J = dJ/dRe u + i dJ/dIm u, for which the
adjoint of a real-linear map d -> alpha d + beta conj(d) is
w -> conj(alpha) w + beta conj(w), and the adjoint of a complex-linear map M
is its conjugate transpose M^H.

Linearisations:
    g: dg = alpha d + beta conj(d),  alpha = gamma - 2 (kappa + i zeta)|u|^2,
       beta = -(kappa + i zeta) u^2  (the source does not depend on u);
    E: complex symmetric, so E^H x = conj(E conj(x));
    parameters: dg/dgamma = u, dg/dkappa = -|u|^2 u, dg/dzeta = -i |u|^2 u;
       dE/dnu = tau K_D E, dE/deta = i tau K_D E with K_D = D_d (+) ... (+) D_1
       the real Kronecker sum (K = (nu + i eta) K_D commutes with K_D).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

from .tensor import mode_product


def _K_D(P, X):
    out = np.zeros_like(X, dtype=np.complex128)
    for mu, D in enumerate(P.Ds, start=1):
        out += mode_product(X, D, mu)
    return out


def _dot(x, y):
    """Re <x, y> = Re sum conj(x) y."""
    return float(np.real(np.vdot(x, y)))


def g_adjoint(P, u, w):
    """(D_u g)^* w."""
    c = P.kappa + 1j * P.zeta
    alpha = P.gamma - 2.0 * c * np.abs(u) ** 2
    beta = -c * u ** 2
    return np.conj(alpha) * w + beta * np.conj(w)


def g_linear(P, u, d):
    """(D_u g) d."""
    c = P.kappa + 1j * P.zeta
    return (P.gamma - 2.0 * c * np.abs(u) ** 2) * d - c * u ** 2 * np.conj(d)


def exp_h(S, tau, x):
    """E^H x = conj(E conj(x)) (E complex symmetric)."""
    return np.conj(S.apply_exp_kron(tau, np.conj(x)))


def forward(S, g, tau, nsteps, u0, t0=0.0):
    """States u_0..u_n and the intermediates (a, v, b, w) of every step."""
    us, inter = [np.asarray(u0, dtype=np.complex128)], []
    t = t0
    for _ in range(nsteps):
        u = us[-1]
        k1 = g(t, u)
        a = u + tau * k1
        v = S.apply_exp_kron(tau, a)
        b = u + 0.5 * tau * k1
        w = S.apply_exp_kron(tau, b)
        us.append(w + 0.5 * tau * g(t + tau, v))
        inter.append((a, v, b, w))
        t += tau
    return us, inter


def loss(S, g, tau, nsteps, u0, u_target, t0=0.0):
    us, _ = forward(S, g, tau, nsteps, u0, t0)
    return 0.5 * float(np.sum(np.abs(us[-1] - u_target) ** 2))


def gradient(S, g, tau, nsteps, u0, u_target, t0=0.0):
    """(J, grad_u0, [dJ/dnu, dJ/deta, dJ/dgamma, dJ/dkappa, dJ/dzeta])."""
    P = S.P
    us, inter = forward(S, g, tau, nsteps, u0, t0)
    lam = us[-1] - u_target
    J = 0.5 * float(np.sum(np.abs(lam) ** 2))
    gp = np.zeros(5)
    for n in reversed(range(nsteps)):
        u = us[n]
        a, v, b, w = inter[n]
        # u' = w + tau/2 g(v)
        lam_w = lam
        lam_gv = 0.5 * tau * lam
        lam_v = g_adjoint(P, v, lam_gv)
        # w = E b, v = E a
        lam_b = exp_h(S, tau, lam_w)
        lam_a = exp_h(S, tau, lam_v)
        # a = u + tau k1, b = u + tau/2 k1, k1 = g(u)
        lam_k1 = tau * lam_a + 0.5 * tau * lam_b
        lam_new = lam_a + lam_b + g_adjoint(P, u, lam_k1)
        # parameters
        gp[0] += tau * (_dot(lam_v, _K_D(P, v)) + _dot(lam_w, _K_D(P, w)))
        gp[1] += tau * (_dot(lam_v, 1j * _K_D(P, v)) + _dot(lam_w, 1j * _K_D(P, w)))
        for z, lz in ((u, lam_k1), (v, lam_gv)):
            gp[2] += _dot(lz, z)
            gp[3] += _dot(lz, -np.abs(z) ** 2 * z)
            gp[4] += _dot(lz, -1j * np.abs(z) ** 2 * z)
        lam = lam_new
    return J, lam, gp
