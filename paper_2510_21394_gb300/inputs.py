"""Seeded synthetic inputs of the FCGLE workloads (shared by tests, bench, smoke).

This module holds no arithmetic of the time-stepping method: only grids,
initial data drawn from seeded generators, and the closed-form continuous
source terms s(t, x) of manufactured exact solutions (they are part of the
problem statement, Eq. FCGLE, not of its discretisation).

Arrays are numpy, shape (n_d, ..., n_1), C order, i.e. vec order with j_1
fastest (Sec. 2, Eq. indexj); complex128 unless stated.

Workloads (recipes; sizes as in the paper's 2D/3D experiments):
* ``gaussian_manufactured``: u = (1+i) e^{-t} exp(-|x|^2) on (-10,10)^d with
  its continuous source s = e^{-t} S_1 + e^{-3t} S_3.
* ``sech_pulse_noise``: sech(|x|) e^{0.5 i x_1} + uniform noise of amplitude
  1e-3 in re and im (PCG64, drawn in vec order).
* ``gaussian_random_phase``: exp(-|x|^2) e^{i pi xi}, xi white noise (PCG64)
  smoothed by a Gaussian of standard deviation ``corr`` physical units (zero
  padded FFT convolution), then standardised.
* ``polynomial_manufactured``: the paper's Example 1,
  u = e^{-i t} prod_mu (1 - x_mu^2)^4 on (-1,1)^d, with its continuous source.
* ``batched_instances``: many independent problems of uneven sizes with
  seeded parameters (square 2D and cubic 3D grids on (-10,10)^d), each started
  from ``gaussian_pulse``.
"""
import math

import numpy as np


def grid(n, a, b):
    h = (b - a) / (n + 1)
    return a + h * np.arange(1, n + 1, dtype=np.float64), h


def mesh(ns, boxes):
    """Coordinates [X_1, ..., X_d] as broadcastable arrays: X_mu has extent
    n_mu on axis d - mu of the tensor shape (n_d, ..., n_1) and 1 elsewhere."""
    d = len(ns)
    out = []
    for mu, (n, (a, b)) in enumerate(zip(ns, boxes)):
        shp = [1] * d
        shp[d - 1 - mu] = n
        out.append(grid(n, a, b)[0].reshape(shp))
    return out


def _shape(ns):
    return tuple(reversed([int(n) for n in ns]))


def _prod(arrs):
    out = arrs[0]
    for a in arrs[1:]:
        out = out * a
    return out


# ---------------------------------------------------------------------------
# Riesz derivatives of the 1D profiles (Sec. 1 definitions)
# ---------------------------------------------------------------------------

def riesz_gaussian(x, alpha):
    """Riesz derivative of exp(-x^2): the inverse Fourier transform of
    -|xi|^alpha sqrt(pi) exp(-xi^2/4), i.e.
    -2^alpha Gamma((1+alpha)/2)/sqrt(pi) * 1F1((1+alpha)/2; 1/2; -x^2).
    Kummer's transformation keeps 1F1 well scaled for large x^2."""
    from scipy.special import hyp1f1, gamma
    a = (1.0 + alpha) / 2.0
    x2 = np.asarray(x, dtype=np.float64) ** 2
    f = np.exp(-x2) * hyp1f1(0.5 - a, 0.5, x2)
    big = x2 > 80.0
    if np.any(big):
        # large-argument form of 1F1(a; 1/2; -x^2) (DLMF 13.7.2 leading terms)
        z = x2[big]
        s = np.zeros_like(z)
        term = np.ones_like(z)
        pref = gamma(0.5) / gamma(0.5 - a)
        for k in range(0, 12):
            s += term
            term = term * (a + k) * (a + 0.5 + k) / ((k + 1) * z)
        f[big] = pref * z ** (-a) * s
    return -(2.0 ** alpha) * gamma(a) / math.sqrt(math.pi) * f


def _poly_coeffs_y():
    """Coefficients c_m of (1-x^2)^4 = y^4 (2-y)^4 in powers of y = 1+x."""
    c = np.zeros(9)
    for j in range(5):
        c[4 + j] = math.comb(4, j) * 2.0 ** (4 - j) * (-1.0) ** j
    return c


def riesz_poly(x, alpha):
    """Riesz derivative of w(x) = (1-x^2)^4 on (-1,1), zero outside, for
    |x| < 1: -1/(2 cos(alpha pi/2)) (D_left + D_right) with the
    Riemann-Liouville power rule D^alpha y^m = Gamma(m+1)/Gamma(m+1-alpha) y^{m-alpha}
    applied in y = 1+x (left) and y = 1-x (right)."""
    from scipy.special import gamma
    x = np.asarray(x, dtype=np.float64)
    c = _poly_coeffs_y()
    yl, yr = 1.0 + x, 1.0 - x
    acc = np.zeros_like(x)
    for m in range(4, 9):
        k = gamma(m + 1.0) / gamma(m + 1.0 - alpha)
        acc += c[m] * k * (yl ** (m - alpha) + yr ** (m - alpha))
    return -acc / (2.0 * math.cos(alpha * math.pi / 2.0))


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def gaussian_manufactured(ns, boxes, alphas, nu, eta, gamma, kappa, zeta):
    """u(t) = (1+i) e^{-t} G, G = exp(-|x|^2); returns (u0, sigmas, [S_1, S_3])
    with s(t, x) = e^{-t} S_1 + e^{-3t} S_3 the continuous source:
    S_1 = (1+i)(-(1+gamma) G - (nu+i eta) sum_mu R_mu(x_mu) prod_{nu!=mu} g(x_nu)),
    S_3 = 2 (1+i)(kappa + i zeta) G^3."""
    X = mesh(ns, boxes)
    gs = [np.exp(-Xm ** 2) for Xm in X]
    G = np.broadcast_to(_prod(gs), _shape(ns))
    lap = np.zeros(_shape(ns))
    for mu in range(len(ns)):
        term = riesz_gaussian(X[mu], alphas[mu])
        for o in range(len(ns)):
            if o != mu:
                term = term * gs[o]
        lap += term
    c = nu + 1j * eta
    S1 = (1 + 1j) * (-(1.0 + gamma) * G - c * lap)
    S3 = 2.0 * (1 + 1j) * (kappa + 1j * zeta) * G ** 3
    u0 = (1 + 1j) * G
    return u0.astype(np.complex128), [-1.0, -3.0], [S1, S3]


def gaussian_exact(ns, boxes, t):
    X = mesh(ns, boxes)
    return np.broadcast_to((1 + 1j) * math.exp(-t) * _prod([np.exp(-Xm ** 2) for Xm in X]), _shape(ns)).copy()


def polynomial_manufactured(ns, alphas, nu, eta, gamma, kappa, zeta):
    """Example 1 of the paper: u = e^{-i t} W, W = prod_mu (1 - x_mu^2)^4 on (-1,1)^d.
    s(t, x) = e^{-i t} S with
    S = (-i - gamma) W - (nu + i eta) sum_mu R_mu(x_mu) prod_{nu != mu} w(x_nu) + (kappa + i zeta) W^3."""
    boxes = [(-1.0, 1.0)] * len(ns)
    X = mesh(ns, boxes)
    ws = [(1.0 - Xm ** 2) ** 4 for Xm in X]
    W = np.broadcast_to(_prod(ws), _shape(ns))
    lap = np.zeros(_shape(ns))
    for mu in range(len(ns)):
        term = riesz_poly(X[mu], alphas[mu])
        for o in range(len(ns)):
            if o != mu:
                term = term * ws[o]
        lap += term
    S = (-1j - gamma) * W - (nu + 1j * eta) * lap + (kappa + 1j * zeta) * W ** 3
    return W.astype(np.complex128), [-1j], [S.astype(np.complex128)]


def polynomial_exact(ns, t):
    X = mesh(ns, [(-1.0, 1.0)] * len(ns))
    return np.broadcast_to(np.exp(-1j * t) * _prod([(1.0 - Xm ** 2) ** 4 for Xm in X]), _shape(ns)).copy()


def sech_pulse_noise(ns, boxes, seed=0, amp=1e-3, k1=0.5):
    X = mesh(ns, boxes)
    r = np.sqrt(sum(Xm ** 2 for Xm in X))
    u = np.broadcast_to((1.0 / np.cosh(r)) * np.exp(1j * k1 * X[0]), _shape(ns))
    rng = np.random.Generator(np.random.PCG64(seed))
    N = u.size
    re = rng.uniform(-amp, amp, N)
    im = rng.uniform(-amp, amp, N)
    return (u + (re + 1j * im).reshape(u.shape)).astype(np.complex128)


def gaussian_random_phase(ns, boxes, seed=1, corr=1.0):
    """exp(-|x|^2) e^{i pi xi}: xi = white noise (PCG64, vec order) convolved
    with a Gaussian of standard deviation ``corr`` (physical units), the noise
    zero-padded by 4 standard deviations on every side (FFT convolution),
    then standardised to zero mean and unit variance."""
    X = mesh(ns, boxes)
    rng = np.random.Generator(np.random.PCG64(seed))
    xi = rng.standard_normal(_shape(ns))
    shape = xi.shape                       # (n_d, ..., n_1)
    hs = [(b - a) / (n + 1) for n, (a, b) in zip(ns, boxes)]
    sig = [corr / h for h in reversed(hs)]  # per axis of `shape`, in grid points
    pads = [int(math.ceil(4.0 * s)) for s in sig]
    full = [n + 2 * p for n, p in zip(shape, pads)]
    buf = np.zeros(full)
    buf[tuple(slice(p, p + n) for p, n in zip(pads, shape))] = xi
    H = np.ones([1] * len(full))
    for ax, (m, s) in enumerate(zip(full, sig)):
        f = np.fft.rfftfreq(m) if ax == len(full) - 1 else np.fft.fftfreq(m)
        hk = np.exp(-2.0 * (math.pi * s * f) ** 2)
        shp = [1] * len(full)
        shp[ax] = hk.size
        H = H * hk.reshape(shp)
    sm = np.fft.irfftn(np.fft.rfftn(buf) * H, s=full)
    xi = sm[tuple(slice(p, p + n) for p, n in zip(pads, shape))]
    xi = (xi - xi.mean()) / xi.std()
    u = np.exp(-sum(Xm ** 2 for Xm in X)) * np.exp(1j * math.pi * xi)
    return u.astype(np.complex128)


def gaussian_pulse(ns, boxes):
    X = mesh(ns, boxes)
    return np.broadcast_to(np.exp(-sum(Xm ** 2 for Xm in X)), _shape(ns)).astype(np.complex128)


def batched_instances(n2=64, n3=32, range2=(128, 768), range3=(48, 160), seed=2):
    """Seeded list of problem specs (dicts: ns, boxes, alphas, nu, eta, gamma,
    kappa, zeta): n2 square 2D grids with n drawn uniformly from range2, then
    n3 cubic 3D grids from range3, on (-10,10)^d.  Per instance the draws are
    taken in this order from one PCG64 stream: n, alpha_mu in [1.1, 1.9]
    (one per direction), nu in [0.5, 2], eta in [-1, 1], zeta in [-1, 1],
    gamma in [0, 1], kappa in [0.5, 2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for d, cnt, (lo, hi) in ((2, n2, range2), (3, n3, range3)):
        for _ in range(cnt):
            n = int(rng.integers(lo, hi + 1))
            alphas = [float(a) for a in rng.uniform(1.1, 1.9, d)]
            nu = float(rng.uniform(0.5, 2.0))
            eta = float(rng.uniform(-1.0, 1.0))
            zeta = float(rng.uniform(-1.0, 1.0))
            gamma = float(rng.uniform(0.0, 1.0))
            kappa = float(rng.uniform(0.5, 2.0))
            out.append(dict(ns=[n] * d, boxes=[(-10.0, 10.0)] * d, alphas=alphas, nu=nu, eta=eta, gamma=gamma,
                            kappa=kappa, zeta=zeta))
    return out
