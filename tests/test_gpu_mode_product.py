"""Kernel-level checks of the raw mode product (fcgle_mode_product).

The eigenvectors are those of the library's own eigensolver, so the checks
use properties that pin them without knowing their order or signs:
* a unit input e_k gives column k of M = Q^T: the rows of the result are
  orthonormal eigenvectors, D q = lam q with lam the Rayleigh quotient
  (D from the oracle's assembly of Eq. Dnalpha);
* the BF16x3 kernel equals the FP64 kernel on random data to split-bf16
  accuracy, and the rotating layout puts the new index slowest.
"""
import numpy as np
import pytest

from oracle import fd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _solver(fc, ns, prec):
    boxes = [(-4.0, 4.0), (-3.0, 3.0), (-5.0, 5.0)][: len(ns)]
    al = [1.3, 1.7, 1.5][: len(ns)]
    return fc.Solver(ns, boxes, al, 1.0, 0.4, 0.5, 1.0, 0.2, precision=prec), boxes, al


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 3e-5)])
def test_unit_vectors_give_eigenvectors(fc, prec, tol):
    ns = [37, 6, 5]                       # p = (40, 8, 8): pads in every direction
    s, boxes, al = _solver(fc, ns, prec)
    p = [(n + 3) // 4 * 4 for n in ns]
    P = fc.fcgle_internal_elems(s.h)
    assert P == int(np.prod(p))
    dt = torch.float64 if prec == "fp64" else torch.float32
    R = P // p[0]
    # X[c][r][k]: row r = 0 carries e_k for k = 0..n1-1 in successive rows r = k
    X = torch.zeros(2, R, p[0], dtype=dt, device="cuda")
    for k in range(ns[0]):
        X[0, k, k] = 1.0
    Y = torch.empty_like(X)
    fc.fcgle_mode_product(s.h, 0, True, X.reshape(-1), Y.reshape(-1))
    s.sync()
    Yn = Y.reshape(2, p[0], R).cpu().numpy().astype(np.float64)
    assert np.all(Yn[1] == 0.0)                       # imaginary plane untouched
    assert np.all(Yn[0, ns[0]:, :] == 0.0)            # padded output rows stay zero
    Q = Yn[0, : ns[0], : ns[0]].T                     # Q[k][i] = (Q^T)[i][k]
    _, h = fd.grid(ns[0], *boxes[0])
    D = fd.D_matrix(ns[0], al[0], h)
    assert np.linalg.norm(Q.T @ Q - np.eye(ns[0])) <= tol * 10
    lam = np.einsum("ki,kl,li->i", Q, D, Q)
    assert np.linalg.norm(D @ Q - Q * lam) <= tol * 10 * np.linalg.norm(D)
    s.close()


def test_bf16x3_matches_fp64_kernel(fc):
    ns = [30, 134, 14]                    # p = (32, 136, 16) in both layouts: 2 i-blocks, 3 k-chunks in direction 2
    s64, _, _ = _solver(fc, ns, "fp64")
    s32, _, _ = _solver(fc, ns, "bf16x3")
    P = fc.fcgle_internal_elems(s64.h)
    assert fc.fcgle_internal_elems(s32.h) == P
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float64, generator=gen)
    for mu in range(3):
        for fwd in (True, False):
            Y64 = torch.empty_like(X)
            Y32 = torch.empty(2 * P, device="cuda", dtype=torch.float32)
            fc.fcgle_mode_product(s64.h, mu, fwd, X, Y64)
            fc.fcgle_mode_product(s32.h, mu, fwd, X.float(), Y32)
            s64.sync()
            s32.sync()
            err = float(torch.linalg.vector_norm(Y32.double() - Y64) / torch.linalg.vector_norm(Y64))
            assert err <= 3e-5, (mu, fwd, err)
    s64.close()
    s32.close()


def _split(x):
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    return torch.cat([hi, lo])


def test_split_io_equals_fp32_io(fc):
    # flags bit 1: the kernel's own input/output format (hi plane pair, then lo)
    ns = [40, 24, 16]
    s, _, _ = _solver(fc, ns, "bf16x3")
    P = fc.fcgle_internal_elems(s.h)
    gen = torch.Generator(device="cuda").manual_seed(1)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float32, generator=gen)
    for mu in range(3):
        Y32 = torch.empty_like(X)
        fc.fcgle_mode_product(s.h, mu, 1, X, Y32)
        Ys = torch.empty(4 * P, device="cuda", dtype=torch.bfloat16)
        fc.fcgle_mode_product(s.h, mu, 1 | 2, _split(X), Ys)
        s.sync()
        y = Ys[: 2 * P].float() + Ys[2 * P:].float()
        err = float(torch.linalg.vector_norm(y - Y32) / torch.linalg.vector_norm(Y32))
        assert err <= 1e-5, (mu, err)
    s.close()


@pytest.mark.parametrize("ns", [[30, 134, 14], [40, 24, 16], [264, 72], [40]])
def test_precise_tf32_product_matches_fp64_kernel(fc, ns):
    """flags bit 2: the precise product of the end transforms (split-TF32 on the
    tensor cores for p <= 256; FP32 on the CUDA cores for d = 1, where R = 1,
    and for p = 264) against the FP64 kernel.  Split-TF32 keeps about 21 significant bits of each operand
    (2^-22 relative) and drops lo.lo (below 2^-22); the tensor core's FP32
    accumulation of the three products over p terms adds the rest.  Measured on
    GB300: at most 2.4e-6 max-elementwise (p = 264, before that size moved to
    the CUDA cores), against 3e-5 for one split-BF16 product; the bound is
    5e-6."""
    s64, _, _ = _solver(fc, ns, "fp64")
    s32, _, _ = _solver(fc, ns, "bf16x3")
    P64 = fc.fcgle_internal_elems(s64.h)
    P32 = fc.fcgle_internal_elems(s32.h)
    assert P64 == P32                     # sizes chosen so that both layouts pad alike
    gen = torch.Generator(device="cuda").manual_seed(2)
    X = torch.randn(2 * P64, device="cuda", dtype=torch.float64, generator=gen)
    for mu in range(len(ns)):
        for fwd in (True, False):
            Y64 = torch.empty_like(X)
            Y32 = torch.empty(2 * P32, device="cuda", dtype=torch.float32)
            fc.fcgle_mode_product(s64.h, mu, fwd, X, Y64)
            fc.fcgle_mode_product(s32.h, mu, int(fwd) | 4, X.float(), Y32)
            s64.sync()
            s32.sync()
            d = Y32.double() - Y64
            err = max(float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(Y64)),
                      float(d.abs().max() / Y64.abs().max()))
            assert err <= 5e-6, (ns, mu, fwd, err)
    with pytest.raises(fc.FcgleError):
        fc.fcgle_mode_product(s32.h, 0, 1 | 2 | 4, X.float(), Y32)
    s64.close()
    s32.close()


_FORCED_CHECK = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2510_21394_gb300 import fcgle
ns = [30, 134, 14]
boxes = [(-4.0, 4.0), (-3.0, 3.0), (-5.0, 5.0)]
al = [1.3, 1.7, 1.5]
pars = (1.0, 0.4, 0.5, 1.0, 0.2)
s64 = fcgle.Solver(ns, boxes, al, *pars, precision="fp64")
s32 = fcgle.Solver(ns, boxes, al, *pars, precision="bf16x3")
P = fcgle.fcgle_internal_elems(s32.h)
gen = torch.Generator(device="cuda").manual_seed(3)
X = torch.randn(2 * P, device="cuda", dtype=torch.float64, generator=gen)
worst = 0.0
for mu in range(3):
    for fwd in (True, False):
        Y64 = torch.empty_like(X)
        Y32 = torch.empty(2 * P, device="cuda", dtype=torch.float32)
        fcgle.fcgle_mode_product(s64.h, mu, fwd, X, Y64)
        fcgle.fcgle_mode_product(s32.h, mu, fwd, X.float(), Y32)
        s64.sync(); s32.sync()
        d = Y32.double() - Y64
        worst = max(worst, float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(Y64)),
                    float(d.abs().max() / Y64.abs().max()))
print("worst", worst)
assert worst <= 3e-5, worst
"""


@pytest.mark.parametrize("cfg", range(6))
def test_every_plain_configuration(fc, cfg):
    """Each ring / tile configuration of the plain product, forced through
    FCGLE_PLAIN_CFG (read once per process, hence a child process), against
    the FP64 kernel; the autotuner only ever runs the fastest one."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, FCGLE_PLAIN_CFG=str(cfg))
    r = subprocess.run([sys.executable, "-c", _FORCED_CHECK.format(root=root)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
