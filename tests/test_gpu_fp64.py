"""FP64 GPU path vs the FP64 oracle (parity bar: 1e-12 relative)."""
import json
import os

import numpy as np
import pytest

from oracle import schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import CONFIG1, PARS, SMALL_CASES, rand_tensor, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("case", range(len(SMALL_CASES)))
@pytest.mark.parametrize("order", [2, 4])
def test_apply_f_parity(fc, case, order):
    ns, boxes, al = SMALL_CASES[case]
    P = tensor.Problem(ns, boxes, al, *PARS.values(), order=order)
    S = tensor.Spectral(P)
    s = fc.Solver(ns, boxes, al, **PARS, fd_order=order, precision="fp64")
    V = rand_tensor(ns, 10 + case)
    v = _dev(V)
    for th in (1e-3, 0.07):
        for func, k in (("inv", 0), ("exp", 0), ("phi", 0), ("phi", 1), ("phi", 2), ("phi", 3), ("phi", 4)):
            kind = {"inv": "inv", "exp": "exp", "phi": "phi"}[func]
            ref = S.apply_f(kind, k, th, V)
            got = _host(s.apply_f(func, k, th, v))
            assert rel(got, ref) <= TOL, (func, k, th, rel(got, ref))
    s.close()


def test_apply_f_in_place_alias(fc):
    ns, boxes, al = SMALL_CASES[1]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    V = rand_tensor(ns, 3)
    s = fc.Solver(ns, boxes, al, **PARS)
    v = _dev(V)
    fc.fcgle_apply_f(s.h, "phi", 2, 0.05, v, v)
    assert rel(_host(v), tensor.Spectral(P).apply_f("phi", 2, 0.05, V)) <= TOL


@pytest.mark.parametrize("scheme", ["lie", "lawson_euler", "lawson_rk2", "etd2rk", "krogstad", "lbdf2", "strang"])
@pytest.mark.parametrize("case", [1, 3, 4])
def test_integrate_parity(fc, scheme, case):
    ns, boxes, al = SMALL_CASES[case]
    pars = dict(PARS)
    P = tensor.Problem(ns, boxes, al, *pars.values())
    u0 = 0.8 * inputs.gaussian_pulse(ns, [(-2.0, 2.0)] * len(ns)) * np.exp(1j * rand_tensor(ns, 4).real)
    src = [] if scheme == "strang" else [0.3 * rand_tensor(ns, 5)]
    sig = [] if scheme == "strang" else [-0.7 + 2.0j]
    g = schemes.Nonlinearity(P, sig, src)
    tau, m = 0.013, 7
    ref = schemes.integrate(tensor.Spectral(P), g, scheme, tau, m, u0, t0=0.2)
    s = fc.Solver(ns, boxes, al, **pars)
    if src:
        s.set_source(sig, [_dev(x) for x in src])
    got = _host(s.integrate(scheme, tau, m, _dev(u0), t0=0.2))
    assert rel(got, ref) <= TOL, rel(got, ref)
    # one-step API agrees with integrate
    if scheme != "lbdf2":
        u = _dev(u0)
        for n in range(m):
            s.step(scheme, tau, 0.2 + n * tau, u)
        assert rel(_host(u), ref) <= TOL
    s.close()


def test_config1_lawson_euler_100_steps(fc):
    """2D 64x64 manufactured Gaussian, Lawson-Euler, T=1, 100 steps, complex128."""
    c = CONFIG1
    P = tensor.Problem(c["ns"], c["boxes"], c["alphas"], *c["pars"].values())
    u0, sig, Ss = inputs.gaussian_manufactured(c["ns"], c["boxes"], c["alphas"], **c["pars"])
    ref = schemes.integrate(tensor.Spectral(P), schemes.Nonlinearity(P, sig, Ss), "lawson_euler", 0.01, 100, u0)
    s = fc.Solver(c["ns"], c["boxes"], c["alphas"], **c["pars"])
    s.set_source(sig, [_dev(x) for x in Ss])
    got = _host(s.integrate("lawson_euler", 0.01, 100, _dev(u0)))
    assert rel(got, ref) <= TOL
    # and the scheme is first order in time around the exact solution: error is O(tau)
    err = schemes.l2_error(P, got, inputs.gaussian_exact(c["ns"], c["boxes"], 1.0))
    assert err < 5e-2


def test_paper_example1_on_gpu(fc):
    """Printed errors of the paper's Example 1 (2D, n = 400) reproduced by the GPU FP64 path."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "example1_errors.json")))
    n, al = 400, [1.2, 1.8]
    pars = dict(nu=1.0, eta=1.0, gamma=3.0, kappa=1.0, zeta=2.0)
    u0, sig, Ss = inputs.polynomial_manufactured([n, n], al, **pars)
    P = tensor.Problem([n, n], [(-1, 1)] * 2, al, *pars.values())
    exact = inputs.polynomial_exact([n, n], 1.0)
    for key, scheme, order in (("lbdf2_fd2", "lbdf2", 2), ("krogstad_fd4", "krogstad", 4)):
        s = fc.Solver([n, n], [(-1.0, 1.0)] * 2, al, **pars, fd_order=order)
        s.set_source(sig, [_dev(x) for x in Ss])
        for m, e in zip(gold[key]["steps"], gold[key]["errors"]):
            got = _host(s.integrate(scheme, 1.0 / m, m, _dev(u0)))
            assert schemes.l2_error(P, got, exact) == pytest.approx(e, rel=1e-4), (key, m)
        s.close()


def test_norm_and_sizes(fc):
    ns, boxes, al = SMALL_CASES[4]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    V = rand_tensor(ns, 9)
    s = fc.Solver(ns, boxes, al, **PARS)
    assert fc.fcgle_sizes(s.h) == (int(np.prod(ns)), int(np.prod(ns)) * 16)
    assert s.norm(_dev(V)) == pytest.approx(np.sqrt(P.cell() * np.sum(np.abs(V) ** 2)), rel=1e-13)
    assert s.launches() > 0


def test_host_buffers_match_device(fc):
    ns, boxes, al = SMALL_CASES[3]
    u0 = inputs.gaussian_pulse(ns, [(-3.0, 3.0)] * 2).astype(np.complex128)
    s = fc.Solver(ns, boxes, al, **PARS)
    dev = _host(s.integrate("krogstad", 0.01, 4, _dev(u0)))
    hin = torch.from_numpy(u0.copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    s.integrate_host("krogstad", 0.01, 4, hin, hout)
    assert np.array_equal(hout.numpy(), dev)
