"""Scalar phi-functions (paper Sec. 4, Eq. phi), FP64 complex.

phi_0(z) = e^z,  phi_l(z) = (phi_{l-1}(z) - 1/(l-1)!) / z,  phi_l(0) = 1/l!.

The recurrence is evaluated as written for |z| >= 1.  For |z| < 1 it cancels
catastrophically, so there the equivalent power series
phi_l(z) = sum_{m>=0} z^m / (m+l)!  (which satisfies the same recurrence
term by term) is summed, 21 terms in Horner form.

Test infrastructure only (see ``oracle/__init__``).
"""
import math
import numpy as np


def phi(ell, z):
    """phi_ell(z) elementwise for a complex array (or scalar) z."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    # power-series branch, Horner form:
    # phi_l(z) = (1/l!) (1 + z/(l+1) (1 + z/(l+2) (1 + ...))); 20 terms leave a
    # remainder below |z|^21/(21+l)! < 2e-20 for |z| < 1
    zs = z[small]
    acc = np.ones(zs.shape, dtype=np.complex128)
    for m in range(20, 0, -1):
        acc = 1.0 + acc * zs / (m + ell)
    out[small] = acc / math.factorial(ell)
    # recurrence branch (Eq. phi, as written)
    zl = z[~small]
    p = np.exp(zl)
    for l in range(1, ell + 1):
        p = (p - 1.0 / math.factorial(l - 1)) / zl
    out[~small] = p
    return out if out.ndim else out[()]
