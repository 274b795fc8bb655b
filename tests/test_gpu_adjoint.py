"""GPU discrete adjoint (Lawson-RK2) vs the FP64 oracle's adjoint and vs
central finite differences of the GPU forward map."""
import numpy as np
import pytest

from oracle import adjoint, schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = [12, 10, 9]
BOXES = [(-3.0, 3.0), (-2.5, 2.5), (-2.0, 2.0)]
AL = [1.5, 1.3, 1.7]
PARS = dict(nu=1.0, eta=0.5, gamma=0.8, kappa=1.2, zeta=0.4)
TAU, M = 0.02, 9


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _case():
    P = tensor.Problem(NS, BOXES, AL, *PARS.values())
    S = tensor.Spectral(P)
    rng = np.random.default_rng(11)
    src = [0.2 * (rng.normal(size=P.shape) + 1j * rng.normal(size=P.shape))]
    g = schemes.Nonlinearity(P, [-0.5 + 1.0j], src)
    u0 = inputs.gaussian_pulse(NS, [(-2.0, 2.0)] * 3) * np.exp(1j * rng.uniform(0, 1, size=P.shape))
    target = 0.9 * adjoint.forward(S, g, TAU, M, u0)[0][-1] + 0.01
    return P, S, g, u0, target, src


def _dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


# split-BF16: the adjoint runs in the eigenbasis with FP32 first / last
# transforms, so the reduced-precision error enters through tau-small terms only
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 2e-4)])
@pytest.mark.parametrize("ckpt", [0, 1, 4])
def test_gradient_matches_oracle(fc, prec, tol, ckpt):
    P, S, g, u0, target, src = _case()
    J, gu, gp = adjoint.gradient(S, g, TAU, M, u0, target)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    s = fc.Solver(NS, BOXES, AL, **PARS, precision=prec)
    s.set_source([-0.5 + 1.0j], [_dev(x, dt) for x in src])
    loss, g_u0, g_par = s.adjoint("lawson_rk2", TAU, M, _dev(u0, dt), _dev(target, dt), ckpt_every=ckpt)
    got = g_u0.cpu().numpy().astype(np.complex128)
    assert loss == pytest.approx(J, rel=tol)
    assert rel(got, gu) <= tol
    np.testing.assert_allclose(g_par, gp, rtol=tol, atol=tol * np.abs(gp).max())
    s.close()


def test_gradient_against_gpu_finite_differences(fc):
    # central differences of J computed by the FP64 GPU forward (fcgle_integrate)
    P, S, g, u0, target, src = _case()
    s = fc.Solver(NS, BOXES, AL, **PARS, precision="fp64")
    s.set_source([-0.5 + 1.0j], [_dev(x, torch.complex128) for x in src])
    tg = _dev(target, torch.complex128)

    def J(u, pars=None):
        if pars is not None:
            s.set_coefficients(*pars)
        uT = s.integrate("lawson_rk2", TAU, M, _dev(u, torch.complex128))
        out = 0.5 * float(torch.sum(torch.abs(uT - tg) ** 2))
        s.set_coefficients(*PARS.values())
        return out
    loss, g_u0, g_par = s.adjoint("lawson_rk2", TAU, M, _dev(u0, torch.complex128), tg, ckpt_every=3)
    rng = np.random.default_rng(5)
    d = rng.normal(size=u0.shape) + 1j * rng.normal(size=u0.shape)
    eps = 1e-6
    fd = (J(u0 + eps * d) - J(u0 - eps * d)) / (2 * eps)
    assert float(np.real(np.vdot(g_u0.cpu().numpy(), d))) == pytest.approx(fd, rel=1e-6)
    base = list(PARS.values())
    for k in range(5):
        h = 1e-6 * max(1.0, abs(base[k]))
        pp, pm = list(base), list(base)
        pp[k] += h
        pm[k] -= h
        fd = (J(u0, pp) - J(u0, pm)) / (2 * h)
        assert g_par[k] == pytest.approx(fd, rel=1e-6, abs=1e-9 * loss), k
    s.close()


def test_autograd_function(fc):
    from paper_2510_21394_gb300.autograd import misfit
    P, S, g, u0, target, src = _case()
    J, gu, gp = adjoint.gradient(S, g, TAU, M, u0, target)
    s = fc.Solver(NS, BOXES, AL, **PARS, precision="fp64")
    s.set_source([-0.5 + 1.0j], [_dev(x, torch.complex128) for x in src])
    u = _dev(u0, torch.complex128).requires_grad_(True)
    p = torch.tensor(list(PARS.values()), dtype=torch.float64, device="cuda", requires_grad=True)
    L = misfit(s, u, p, _dev(target, torch.complex128), tau=TAU, nsteps=M, ckpt_every=4)
    (2.0 * L).backward()
    assert float(L) == pytest.approx(J, rel=1e-10)
    assert np.linalg.norm(u.grad.cpu().numpy() - 2 * gu) <= 1e-10 * np.linalg.norm(2 * gu)
    np.testing.assert_allclose(p.grad.cpu().numpy(), 2 * gp, rtol=1e-9)
    s.close()
