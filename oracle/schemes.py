"""Time integrators, FP64, in their vector form (paper Sec. 4), built on O2.

ODE (Eq. ODEs): u' = K u + g(t, u) with (Sec. 2)
    g(t, u) = gamma u - (kappa + i zeta) |u|^2 u + s(t),
and the source written as s(t) = sum_k exp(sigma_k t) S_k (sigma_k complex),
which covers every manufactured source used here.

Schemes (each step maps (t_n, u_n) -> u_{n+1}):
* ``lie``      linearly-implicit (backward-forward) Euler (Eq. lbdf2-v, first
               step): u_{n+1} = (I - tau K)^{-1}(u_n + tau g(t_n, u_n)).
* ``lbdf2``    linearised BDF2 (Eq. lbdf2-v), first step by ``lie``.
* ``strang``   Strang splitting (Eq. Strang) with the exact nonlinear flow
               (Sec. 4) and exp(tau K); no source.
* ``krogstad`` Krogstad's fourth-order exponential RK (Eq. krogstad-v).
* ``lawson_euler``, ``lawson_rk2``, ``etd2rk``: not in the paper; standard
               forms taken here: Lawson-Euler u' = e^{tau K}(u + tau g(t, u));
               Heun-based Lawson k1 = g(t, u), v = e^{tau K}(u + tau k1),
               u' = e^{tau K}(u + tau/2 k1) + tau/2 g(t + tau, v); Cox-Matthews
               ETD2RK a = u + tau phi_1(tau K) f, u' = a + tau phi_2(tau K)
               (g(t + tau, a) - g(t, u)), f = K u + g(t, u).

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

from .tensor import K_apply
from .phi import phi


class Nonlinearity:
    def __init__(self, P, sigmas=(), Ss=()):
        self.P = P
        self.sigmas = [complex(s) for s in sigmas]
        self.Ss = [np.asarray(S, dtype=np.complex128) for S in Ss]

    def source(self, t):
        s = np.zeros(self.P.shape, dtype=np.complex128)
        for sig, S in zip(self.sigmas, self.Ss):
            s = s + np.exp(sig * t) * S
        return s

    def __call__(self, t, u):
        P = self.P
        return (P.gamma * u - (P.kappa + 1j * P.zeta) * (np.abs(u) ** 2) * u
                + self.source(t))


def lie_step(S, g, tau, t, u):
    return S.apply_f("inv", 0, tau, u + tau * g(t, u))


def lbdf2_step(S, g, tau, t, u, u_prev):
    """One step n -> n+1 of Eq. lbdf2-v (n >= 1); t = t_n."""
    u2 = 2.0 * u - u_prev
    rhs = (4.0 / 3.0) * u - (1.0 / 3.0) * u_prev + (2.0 * tau / 3.0) * g(t + tau, u2)
    return S.apply_f("inv", 0, 2.0 * tau / 3.0, rhs)


def exact_flow(P, t, w):
    """phi_t(w) = exp(t gamma - (kappa+i zeta)/(2 kappa) log(1 + 2 t phi_1(2 gamma t) kappa |w|^2)) w."""
    p1 = complex(phi(1, 2.0 * P.gamma * t)).real
    arg = 1.0 + 2.0 * t * p1 * P.kappa * np.abs(w) ** 2
    return np.exp(t * P.gamma - (P.kappa + 1j * P.zeta) / (2.0 * P.kappa) * np.log(arg)) * w


def strang_step(S, g, tau, t, u):
    P = S.P
    return exact_flow(P, tau / 2, S.apply_exp_kron(tau, exact_flow(P, tau / 2, u)))


def krogstad_step(S, g, tau, t, u):
    """Eq. krogstad-v with f_n = K u_n + g(t_n, u_n), d_ni = g(t_n + c_i tau, u_ni) - g(t_n, u_n)."""
    P = S.P
    gn = g(t, u)
    fn = K_apply(P, u) + gn
    ph = lambda l, th, v: S.apply_f("phi", l, th, v)
    u2 = u + (tau / 2) * ph(1, tau / 2, fn)
    d2 = g(t + tau / 2, u2) - gn
    u3 = u + (tau / 2) * ph(1, tau / 2, fn) + tau * ph(2, tau / 2, d2)
    d3 = g(t + tau / 2, u3) - gn
    u4 = u + tau * ph(1, tau, fn) + 2 * tau * ph(2, tau, d3)
    d4 = g(t + tau, u4) - gn
    return (u + tau * ph(1, tau, fn)
            + tau * ph(2, tau, 2 * d2 + 2 * d3 - d4)
            + tau * ph(3, tau, -4 * d2 - 4 * d3 + 4 * d4))


def lawson_euler_step(S, g, tau, t, u):
    """u_{n+1} = exp(tau K)(u_n + tau g(t_n, u_n))."""
    return S.apply_exp_kron(tau, u + tau * g(t, u))


def lawson_rk2_step(S, g, tau, t, u):
    """Heun applied to w = exp(-tK) u:
    k1 = g(t_n, u_n); v = E(u_n + tau k1);
    u_{n+1} = E(u_n + tau/2 k1) + tau/2 g(t_n + tau, v),  E = exp(tau K)."""
    k1 = g(t, u)
    v = S.apply_exp_kron(tau, u + tau * k1)
    return S.apply_exp_kron(tau, u + (tau / 2) * k1) + (tau / 2) * g(t + tau, v)


def etd2rk_step(S, g, tau, t, u):
    """Cox-Matthews ETD2RK:
    a = exp(tau K) u_n + tau phi_1(tau K) g(t_n, u_n);
    u_{n+1} = a + tau phi_2(tau K)(g(t_n + tau, a) - g(t_n, u_n))."""
    gn = g(t, u)
    a = S.apply_f("exp", 0, tau, u) + tau * S.apply_f("phi", 1, tau, gn)
    return a + tau * S.apply_f("phi", 2, tau, g(t + tau, a) - gn)


ONE_STEP = {
    "lie": lie_step,
    "lawson_euler": lawson_euler_step,
    "lawson_rk2": lawson_rk2_step,
    "etd2rk": etd2rk_step,
    "krogstad": krogstad_step,
    "strang": strang_step,
}


def integrate(S, g, scheme, tau, nsteps, u0, t0=0.0):
    """Advance u0 by nsteps constant steps of size tau."""
    u = np.asarray(u0, dtype=np.complex128)
    t = t0
    if scheme == "lbdf2":
        if nsteps == 0:
            return u
        u_prev, u = u, lie_step(S, g, tau, t, u)
        t += tau
        for _ in range(nsteps - 1):
            u_prev, u = u, lbdf2_step(S, g, tau, t, u, u_prev)
            t += tau
        return u
    step = ONE_STEP[scheme]
    for _ in range(nsteps):
        u = step(S, g, tau, t, u)
        t += tau
    return u


def l2_error(P, u, v):
    """Discrete L^2 norm of u - v: (prod_mu h_mu sum_j |e_j|^2)^{1/2} (Sec. 4)."""
    return float(np.sqrt(P.cell() * np.sum(np.abs(u - v) ** 2)))
