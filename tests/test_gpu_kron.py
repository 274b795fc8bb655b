"""The Kronecker-product form of the exponential on the tensor cores
(Eqs. Neudecker, Neudeckerd): V x_1 E_1 ... x_d E_d with complex
E_mu = exp(theta A_mu), as split-BF16 complex mode products (one N = 128
product with Re E over both planes, two N = 64 products with Im E).

* fcgle_apply_f(EXP) in this form against the oracle's Kronecker-product
  exponential (apply_exp_kron) and its Tucker-form exponential, on distinct
  sizes per direction with ragged tails, d = 1, 2, 3, several i-blocks and
  k-chunks;
* Lawson-Euler, Lawson-RK2 and Strang, whose only linear operator is
  e^{tau K}, in this form against the oracle schemes;
* at a larger size, a few steps of each against the Tucker form of the same
  handle type.

Tolerance: each complex product rounds both operands to 16 significant bits
(split-BF16, about 2^-17 relative each) and d of them chain: 1e-4 relative
for the small cases, as for the Tucker form.
"""
import numpy as np
import pytest

from oracle import schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import PARS, SMALL_CASES, rand_tensor, rel, rel_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


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


CASES = SMALL_CASES + [([300, 9], [(-5.0, 5.0)] * 2, [1.3, 1.6]), ([20, 257, 6], [(-5.0, 5.0)] * 3, [1.3, 1.6, 1.8])]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_apply_exp_kron_matches_oracle(fc, case):
    ns, boxes, al = CASES[case]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    S = tensor.Spectral(P)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    s.set_exp_form("kron")
    V = rand_tensor(ns, 40 + case).astype(np.complex64).astype(np.complex128)
    for th in (1e-3, 0.07):
        ref_k = S.apply_exp_kron(th, V)
        for func, k in (("exp", 0), ("phi", 0)):
            got = _host(s.apply_f(func, k, th, _dev(V)))
            assert rel(got, ref_k) <= TOL, (ns, th, func, rel(got, ref_k))
        assert rel(ref_k, S.apply_f("exp", 0, th, V)) <= 1e-12   # the two forms of the oracle agree
    s.sync()
    s.close()


@pytest.mark.parametrize("scheme", ["lawson_euler", "lawson_rk2", "strang"])
@pytest.mark.parametrize("case", [1, 3, 4])
def test_kron_schemes_match_oracle(fc, scheme, case):
    ns, boxes, al = SMALL_CASES[case]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    u0 = 0.8 * inputs.gaussian_pulse(ns, [(-2.0, 2.0)] * len(ns)) * np.exp(1j * rand_tensor(ns, 4).real)
    u0 = u0.astype(np.complex64).astype(np.complex128)
    src = [] if scheme == "strang" else [0.3 * rand_tensor(ns, 5).astype(np.complex64).astype(np.complex128)]
    sig = [] if scheme == "strang" else [-0.7 + 2.0j]
    g = schemes.Nonlinearity(P, sig, src)
    tau, m = 0.013, 7
    ref = schemes.integrate(tensor.Spectral(P), g, scheme, tau, m, u0, t0=0.2)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    s.set_exp_form("kron")
    if src:
        s.set_source(sig, [_dev(x) for x in src])
    got = _host(s.integrate(scheme, tau, m, _dev(u0), t0=0.2))
    s.sync()
    assert rel(got, ref) <= TOL, (scheme, ns, rel(got, ref))
    s.close()


@pytest.mark.parametrize("scheme", ["lawson_euler", "lawson_rk2", "strang"])
def test_kron_form_against_tucker_form_128cube(fc, scheme):
    ns, boxes, al = [128, 120, 136], [(-10.0, 10.0)] * 3, [1.2, 1.5, 1.8]
    u0 = _dev(inputs.gaussian_random_phase(ns, boxes, seed=1))
    a = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    b = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    b.set_exp_form("kron")
    ua = a.integrate(scheme, 1e-3, 10, u0)
    ub = b.integrate(scheme, 1e-3, 10, u0)
    a.sync()
    b.sync()
    assert rel_dev(ub, ua.to(torch.complex128)) <= 1e-4
    a.close()
    b.close()


def test_exp_form_rejects_unknown_values(fc):
    ns, boxes, al = SMALL_CASES[0]
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    with pytest.raises(fc.FcgleError) as e:
        fc.fcgle_set_exp_form(s.h, 2)
    assert e.value.status == fc.FCGLE_ERR_INVALID_ARG
    s.close()
