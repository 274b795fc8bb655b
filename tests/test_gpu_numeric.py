"""Non-finite detection and the device spectral scalars.

* A NaN or an Inf in a result state is reported as FCGLE_ERR_NUMERIC by the
  next synchronising call, in both precisions, and the handle stays usable.
* The spectral scalars f(theta lam) (Eq. phi for phi_k; Sec. 3.2 for the
  diagonal of f(Lam)) as the kernels evaluate them, against the FP64 oracle's
  scalar functions, on both sides of the |z| = 1 switch between the power
  series and the recurrence.

FP32 tolerance of the BF16X3 scalars, from the arithmetic: z is formed in FP32
(|dz| <= 3 ulp |z|, so |df/f| <= |z f'/f| 1.8e-7 <= 1e-6 for |z| <= 4.5 on
the rays used); the series branch (|z| < 1) is a 10-term Horner sum (a few ulp);
the recurrence branch (|z| >= 1) divides phi_{l-1} - 1/(l-1)! by z, and each
level amplifies the relative error by |phi_{l-1}| / |phi_l z| <= 4 there, so
phi_3 carries at most ~3 x 4^2 ulp ~ 3e-6 and phi_4 ~4 x that.  The FP64
handle evaluates in FP64 (the recurrence loses at most 4^4 ulp ~ 6e-14).
"""
import math

import numpy as np
import pytest

from oracle import phi as ophi
from oracle import tensor
from helpers import PARS, SMALL_CASES, rand_tensor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = {"inv": 2e-6, "exp": 2e-6, 0: 2e-6, 1: 2e-6, 2: 4e-6, 3: 6e-6, 4: 3e-5}
TOL64 = 1e-12


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _eig_sums(theta, nu, eta):
    """Real eigenvalue sums s <= 0 with |z| = |theta (nu + i eta) s| from 1e-6 to
    4.5, dense around |z| = 1 (both sides), plus s = 0."""
    w = abs(theta * complex(nu, eta))
    az = np.concatenate([np.logspace(-6, math.log10(4.5), 60), 1.0 + np.array([-1e-3, -1e-5, 0.0, 1e-5, 1e-3]),
                         np.linspace(0.9, 1.1, 21)])
    return np.concatenate([[0.0], -np.sort(az) / w])


def _oracle(func, k, z):
    if func == "inv":
        return 1.0 / (1.0 - z)
    if func == "exp" or k == 0:
        return np.exp(z)
    return ophi.phi(k, z)


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
@pytest.mark.parametrize("fk", [("inv", 0), ("exp", 0), ("phi", 0), ("phi", 1), ("phi", 2), ("phi", 3),
                                ("phi", 4)])
def test_spectral_scalars_match_oracle(fc, prec, fk):
    func, k = fk
    ns, boxes, al = SMALL_CASES[0]
    pars = dict(PARS)
    s = fc.Solver(ns, boxes, al, **pars, precision=prec)
    theta = 1e-3
    sv = _eig_sums(theta, pars["nu"], pars["eta"])
    forms = [0, 1] if (prec == "bf16x3" and func == "phi" and 1 <= k <= 3) else [0]
    for form in forms:
        got = np.array(fc.fcgle_spectral_scalars(s.h, func, k, theta, sv, form))
        if prec == "bf16x3":
            s32 = sv.astype(np.float32).astype(np.float64)   # the kernels hold s in FP32
            ref = _oracle(func, k, theta * complex(pars["nu"], pars["eta"]) * s32)
            tol = TOL32[func if func != "phi" else k]
        else:
            ref = _oracle(func, k, theta * complex(pars["nu"], pars["eta"]) * sv)
            tol = TOL64
        err = np.abs(got - ref) / np.abs(ref)
        assert err.max() <= tol, (prec, func, k, form, float(err.max()), float(sv[np.argmax(err)]))
    s.close()


def test_spectral_scalars_reject_bad_arguments(fc):
    ns, boxes, al = SMALL_CASES[0]
    s = fc.Solver(ns, boxes, al, **PARS, precision="fp64")
    for args in (("phi", 5, 1e-3, [1.0], 0), ("phi", 1, 1e-3, [float("nan")], 0), ("phi", 1, 1e-3, [1.0], 1)):
        with pytest.raises(fc.FcgleError) as e:
            fc.fcgle_spectral_scalars(s.h, *args)
        assert e.value.status == fc.FCGLE_ERR_INVALID_ARG
    s.close()


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_state_is_reported(fc, prec, bad):
    ns, boxes, al = SMALL_CASES[4]
    dt = torch.complex64 if prec == "bf16x3" else torch.complex128
    s = fc.Solver(ns, boxes, al, **PARS, precision=prec)
    clean = torch.from_numpy(0.3 * rand_tensor(ns, 3)).to(dt).cuda()
    u0 = clean.clone()
    u0.view(-1)[17] = complex(bad, 0.0)
    out = s.integrate("etd2rk", 1e-3, 3, u0)
    with pytest.raises(fc.FcgleError) as e:
        s.sync()
    assert e.value.status == fc.FCGLE_ERR_NUMERIC
    # the report clears the word; a clean run afterwards synchronises without error
    out = s.integrate("etd2rk", 1e-3, 3, clean)
    s.sync()
    assert torch.isfinite(torch.view_as_real(out)).all()
    # apply_f output and the host-buffer entry point report it too
    s.apply_f("phi", 1, 1e-3, u0)
    with pytest.raises(fc.FcgleError) as e:
        s.sync()
    assert e.value.status == fc.FCGLE_ERR_NUMERIC
    hin = u0.cpu().pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    with pytest.raises(fc.FcgleError) as e:
        s.integrate_host("lie", 1e-3, 2, hin, hout)
    assert e.value.status == fc.FCGLE_ERR_NUMERIC
    s.sync()
    s.close()


def test_nonfinite_instance_of_a_batch(fc):
    specs = [dict(ns=[n] * 2, boxes=[(-5.0, 5.0)] * 2, alphas=[1.4, 1.6], **PARS) for n in (24, 40)]
    b = fc.Batch(specs, precision="bf16x3")
    u0 = [torch.from_numpy(0.3 * rand_tensor(sp["ns"], 5)).to(torch.complex64).cuda() for sp in specs]
    u0[1].view(-1)[3] = complex(float("nan"), 0.0)
    b.integrate("etd2rk", 1e-3, 3, u0, use_graph=True)
    fc.fcgle_sync(b.instance(0))
    with pytest.raises(fc.FcgleError) as e:
        fc.fcgle_sync(b.instance(1))
    assert e.value.status == fc.FCGLE_ERR_NUMERIC
    b.close()
