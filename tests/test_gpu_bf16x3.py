"""Split-BF16 tensor-core path (complex64 storage) vs the FP64 oracle.

Tolerances follow from the arithmetic: each mode product rounds both
operands to 16 significant bits (x = x_hi + x_lo, |x - x_hi - x_lo| <= 2^-17 |x|)
and drops x_lo * M_lo, so one mode product has a relative error of a few
2^-17 ~ 8e-6 (plus FP32 storage, 6e-8); f(theta K) v chains 2d of them.
"""
import numpy as np
import pytest

from oracle import schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import PARS, SMALL_CASES, rand_tensor, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_APPLY = 1e-4      # 2d <= 6 split-bf16 mode products
TOL_INTEGRATE = 1e-4  # a few steps of a scheme at small sizes


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def test_identity_roundtrip(fc):
    # phi_0(0 K) = I: forward then backward Tucker must reproduce v to bf16x3 accuracy
    ns, boxes, al = SMALL_CASES[4]
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    V = rand_tensor(ns, 1).astype(np.complex64).astype(np.complex128)
    got = _host(s.apply_f("inv", 0, 0.0, _dev(V)))
    s.sync()
    assert rel(got, V) <= 3e-5


@pytest.mark.parametrize("case", range(len(SMALL_CASES)))
def test_apply_f_parity(fc, case):
    ns, boxes, al = SMALL_CASES[case]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    S = tensor.Spectral(P)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    V = rand_tensor(ns, 20 + case)
    v = _dev(V)
    V32 = V.astype(np.complex64).astype(np.complex128)
    for th in (1e-3, 0.07):
        for func, k in (("inv", 0), ("exp", 0), ("phi", 0), ("phi", 1), ("phi", 2), ("phi", 3), ("phi", 4)):
            ref = S.apply_f(func, k, th, V32)
            got = _host(s.apply_f(func, k, th, v))
            assert rel(got, ref) <= TOL_APPLY, (func, k, th, rel(got, ref))
    s.sync()
    s.close()


@pytest.mark.parametrize("scheme", ["lie", "lawson_euler", "lawson_rk2", "etd2rk", "krogstad", "lbdf2", "strang"])
def test_integrate_parity(fc, scheme):
    ns, boxes, al = SMALL_CASES[4]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    u0 = (0.8 * inputs.gaussian_pulse(ns, [(-2.0, 2.0)] * 3) * np.exp(1j * rand_tensor(ns, 4).real))
    u0 = u0.astype(np.complex64).astype(np.complex128)
    src = [] if scheme == "strang" else [0.3 * rand_tensor(ns, 5).astype(np.complex64).astype(np.complex128)]
    sig = [] if scheme == "strang" else [-0.7 + 2.0j]
    g = schemes.Nonlinearity(P, sig, src)
    tau, m = 0.013, 7
    ref = schemes.integrate(tensor.Spectral(P), g, scheme, tau, m, u0, t0=0.2)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    if src:
        s.set_source(sig, [_dev(x) for x in src])
    got = _host(s.integrate(scheme, tau, m, _dev(u0), t0=0.2))
    s.sync()
    assert rel(got, ref) <= TOL_INTEGRATE, rel(got, ref)
    s.close()


def test_large_mode_sizes(fc):
    # p > 128 and p > 256 exercise several i-blocks and k-chunks of the kernel
    for ns in ([300, 9], [20, 257, 6]):
        boxes = [(-5.0, 5.0)] * len(ns)
        al = [1.3, 1.6, 1.8][: len(ns)]
        P = tensor.Problem(ns, boxes, al, *PARS.values())
        V = rand_tensor(ns, 7).astype(np.complex64).astype(np.complex128)
        s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
        got = _host(s.apply_f("phi", 1, 0.01, _dev(V)))
        s.sync()
        assert rel(got, tensor.Spectral(P).apply_f("phi", 1, 0.01, V)) <= TOL_APPLY
        s.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_zero_steps_return_the_input(fc, prec):
    """nsteps = 0 is the identity on the state (pack then unpack, no step)."""
    ns, boxes, al = SMALL_CASES[4]
    dt = torch.complex64 if prec == "bf16x3" else torch.complex128
    s = fc.Solver(ns, boxes, al, **PARS, precision=prec)
    u0 = torch.from_numpy(rand_tensor(ns, 8)).to(dt).cuda()
    for scheme in ("krogstad", "lbdf2", "strang"):
        out = s.integrate(scheme, 1e-3, 0, u0)
        s.sync()
        assert torch.equal(out, u0)
    s.close()


def test_large_extents_many_blocks_and_chunks(fc):
    """2D 2048 x 1536: 16 and 12 i-blocks, 32 and 24 k-chunks per unit; the
    plain product runs in the autotuner's choice for these shapes, and the
    precise end transforms on the CUDA cores (p > 256)."""
    ns = [2048, 1536]
    boxes = [(-20.0, 20.0), (-15.0, 15.0)]
    al = [1.3, 1.7]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    S = tensor.Spectral(P)
    V = rand_tensor(ns, 12).astype(np.complex64).astype(np.complex128)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    for func, k in (("phi", 1), ("inv", 0)):
        got = _host(s.apply_f(func, k, 1e-3, _dev(V)))
        assert rel(got, S.apply_f(func, k, 1e-3, V)) <= TOL_APPLY
    u0 = (0.8 * inputs.gaussian_pulse(ns, boxes)).astype(np.complex64).astype(np.complex128)
    g = schemes.Nonlinearity(P)
    ref = schemes.integrate(S, g, "etd2rk", 1e-3, 2, u0)
    got = _host(s.integrate("etd2rk", 1e-3, 2, _dev(u0)))
    s.sync()
    assert rel(got, ref) <= TOL_INTEGRATE
    s.close()
