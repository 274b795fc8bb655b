"""Shared helpers of the test-suite: workload definitions and conversions."""
import numpy as np

CONFIG1 = dict(ns=[64, 64], boxes=[(-10.0, 10.0)] * 2, alphas=[1.5, 1.5],
               pars=dict(nu=1.0, eta=0.5, gamma=1.0, kappa=1.0, zeta=0.5))
CONFIG2 = dict(ns=[1023, 1024], boxes=[(-20.0, 20.0)] * 2, alphas=[1.3, 1.7],
               pars=dict(nu=1.0, eta=1.0, gamma=0.5, kappa=1.0, zeta=-1.0))
CONFIG3 = dict(ns=[256, 256, 256], boxes=[(-10.0, 10.0)] * 3, alphas=[1.2, 1.5, 1.8],
               pars=dict(nu=1.0, eta=0.5, gamma=1.0, kappa=1.0, zeta=0.5))

SMALL_CASES = [
    # (ns, boxes, alphas): distinct sizes per direction, several tiles plus ragged tails
    ([7, 9], [(-1.0, 1.0), (-3.0, 2.0)], [1.2, 1.8]),
    ([5, 6, 8], [(-2.0, 2.0), (-1.0, 3.0), (-1.5, 1.5)], [1.2, 1.8, 1.5]),
    ([11], [(-1.0, 1.0)], [1.4]),
    ([70, 45], [(-5.0, 5.0), (-4.0, 4.0)], [1.3, 1.7]),
    ([33, 20, 29], [(-4.0, 4.0), (-3.0, 3.0), (-5.0, 5.0)], [1.5, 1.2, 1.9]),
    ([130, 3], [(-6.0, 6.0), (-1.0, 1.0)], [1.6, 1.4]),
]

PARS = dict(nu=1.0, eta=0.6, gamma=0.5, kappa=1.0, zeta=-0.3)


def rand_tensor(ns, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(ns))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel_norm(a, b):
    """Norm-wise relative error ||a - b||_2 / ||b||_2."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rel_max(a, b):
    """Max-elementwise relative error ||a - b||_inf / ||b||_inf: an error confined
    to a few entries (a ragged tail, a padding row) is not diluted by the rest."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def rel(a, b):
    """The larger of the norm-wise and the max-elementwise relative errors; every
    parity comparison of the GPU tests holds both to its tolerance."""
    return max(rel_norm(a, b), rel_max(a, b))


def rel_dev(a, b):
    """rel() for two CUDA tensors (a is promoted to b's dtype), without a host copy."""
    import torch
    a = a.to(b.dtype)
    d = a - b
    nrm = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(b))
    mx = float(d.abs().max() / b.abs().max())
    return max(nrm, mx)
