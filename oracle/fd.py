"""Spatial semidiscretisation (paper Sec. 2), FP64.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np


def grid(n, a, b):
    """Interior points x^j = a + j h, j = 1..n, h = (b-a)/(n+1)  (Sec. 2)."""
    h = (b - a) / (n + 1)
    return a + h * np.arange(1, n + 1, dtype=np.float64), h


def g_coeffs(alpha, n):
    """FD2 coefficients g_k^(alpha), k = 0..n-1, by the recurrence of Sec. 2:

    g_0 = Gamma(alpha+1) / Gamma(alpha/2+1)^2,
    g_k = (1 - (alpha+1)/(alpha/2+k)) g_{k-1}.
    """
    from math import gamma
    g = np.empty(n, dtype=np.float64)
    g[0] = gamma(alpha + 1.0) / gamma(alpha / 2.0 + 1.0) ** 2
    for k in range(1, n):
        g[k] = (1.0 - (alpha + 1.0) / (alpha / 2.0 + k)) * g[k - 1]
    return g


def g_coeffs_fd4(alpha, n):
    """FD4 coefficients (Sec. 2, Eq. FD4): 4/3 g_k for odd k,
    4/3 g_k - (1/3) g_{k/2} / 2^alpha for even k."""
    g = g_coeffs(alpha, n)
    gc = (4.0 / 3.0) * g
    for k in range(0, n, 2):
        gc[k] -= (1.0 / 3.0) * g[k // 2] / 2.0 ** alpha
    return gc


def D_matrix(n, alpha, h, order=2):
    """D_n^alpha = -h^{-alpha} toeplitz(g_0 .. g_{n-1})  (Eq. Dnalpha)."""
    g = g_coeffs(alpha, n) if order == 2 else g_coeffs_fd4(alpha, n)
    idx = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    return -(h ** (-alpha)) * g[idx]
