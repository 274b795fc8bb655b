"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the bench uses (one fcgle_integrate call of all steps).

At these sizes the FP64 oracle cannot run the whole horizon in test time, so
each case (1) pins the FP64 GPU path to the oracle on a sampled window at full
size (<= 1e-12 relative) and (2) holds the split-BF16 tensor-core path to the
FP64 GPU path at the final time T (<= 1e-5 relative, the stated tolerance of
the reduced-precision form)."""
import numpy as np
import pytest

from helpers import CONFIG2, CONFIG3, rel, rel_dev
from oracle import schemes, tensor
from paper_2510_21394_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL64 = 1e-12
TOL_TC = 1e-5


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _rel_dev(a, b):
    torch.cuda.synchronize()
    return rel_dev(a, b)


@pytest.mark.parametrize("scheme", ["lie", "etd2rk"])
def test_config2_1023x1024_500_steps(fc, scheme):
    """2D 1023x1024 on (-20,20)^2, sech pulse + noise, tau = 1e-3, 500 steps."""
    c = CONFIG2
    u0 = inputs.sech_pulse_noise(c["ns"], c["boxes"], seed=0)
    s64 = fc.Solver(c["ns"], c["boxes"], c["alphas"], **c["pars"], precision="fp64")
    s32 = fc.Solver(c["ns"], c["boxes"], c["alphas"], **c["pars"], precision="bf16x3")
    v64 = torch.from_numpy(u0).cuda()
    # (1) FP64 GPU vs oracle, first 3 steps at full size
    P = tensor.Problem(c["ns"], c["boxes"], c["alphas"], *c["pars"].values())
    ref = schemes.integrate(tensor.Spectral(P), schemes.Nonlinearity(P), scheme, 1e-3, 3, u0)
    got = s64.integrate(scheme, 1e-3, 3, v64)
    torch.cuda.synchronize()
    assert rel(got.cpu().numpy(), ref) <= TOL64
    # the split-BF16 path on the same window, against the oracle directly
    got32 = s32.integrate(scheme, 1e-3, 3, v64.to(torch.complex64))
    torch.cuda.synchronize()
    assert rel(got32.cpu().numpy().astype(np.complex128), ref) <= TOL_TC
    # (2) split-BF16 vs FP64 GPU at T = 0.5
    a = s64.integrate(scheme, 1e-3, 500, v64)
    b = s32.integrate(scheme, 1e-3, 500, v64.to(torch.complex64))
    assert _rel_dev(b, a) <= TOL_TC
    assert torch.isfinite(torch.view_as_real(a)).all()
    s64.close()
    s32.close()


def test_config3_256cube_krogstad_200_steps(fc):
    """3D 256^3 on (-10,10)^3, Gaussian x smoothed random phase, Krogstad, tau = 1e-3, 200 steps."""
    c = CONFIG3
    u0 = inputs.gaussian_random_phase(c["ns"], c["boxes"], seed=1)
    s64 = fc.Solver(c["ns"], c["boxes"], c["alphas"], **c["pars"], precision="fp64")
    s32 = fc.Solver(c["ns"], c["boxes"], c["alphas"], **c["pars"], precision="bf16x3")
    v64 = torch.from_numpy(u0).cuda()
    # (1) FP64 GPU vs oracle, one step at full size
    P = tensor.Problem(c["ns"], c["boxes"], c["alphas"], *c["pars"].values())
    ref = schemes.integrate(tensor.Spectral(P), schemes.Nonlinearity(P), "krogstad", 1e-3, 1, u0)
    got = s64.integrate("krogstad", 1e-3, 1, v64)
    torch.cuda.synchronize()
    assert rel(got.cpu().numpy(), ref) <= TOL64
    # the split-BF16 path on the same step, against the oracle directly
    got32 = s32.integrate("krogstad", 1e-3, 1, v64.to(torch.complex64))
    torch.cuda.synchronize()
    assert rel(got32.cpu().numpy().astype(np.complex128), ref) <= TOL_TC
    del ref, got, got32
    # (2) split-BF16 vs FP64 GPU at T = 0.2
    a = s64.integrate("krogstad", 1e-3, 200, v64)
    b = s32.integrate("krogstad", 1e-3, 200, v64.to(torch.complex64))
    assert _rel_dev(b, a) <= TOL_TC
    s64.close()
    s32.close()


def test_config4_batched_96_instances(fc):
    """96 uneven instances (64 2D 128^2..768^2, 32 3D 48^3..160^3), ETD2RK, tau = 1e-3,
    100 steps, one CUDA graph per step; every sixth instance against FP64."""
    specs = inputs.batched_instances()
    assert len(specs) == 96
    b32 = fc.Batch(specs, precision="bf16x3")
    u0 = [torch.from_numpy(inputs.gaussian_pulse(sp["ns"], sp["boxes"])).cuda() for sp in specs]
    o32 = b32.integrate("etd2rk", 1e-3, 100, [x.to(torch.complex64) for x in u0], use_graph=True)
    torch.cuda.synchronize()
    assert b32.launches()[1] == 100
    # grouped persistent launches (one per phase over all 96 instances): bitwise the same
    og = b32.integrate("etd2rk", 1e-3, 100, [x.to(torch.complex64) for x in u0], grouped=True)
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(o32, og))
    sample = list(range(0, 96, 6))
    b64 = fc.Batch([specs[i] for i in sample], precision="fp64")
    o64 = b64.integrate("etd2rk", 1e-3, 100, [u0[i] for i in sample])
    errs = [_rel_dev(o32[i], o64[k]) for k, i in enumerate(sample)]
    assert max(errs) <= TOL_TC, errs
    # every instance finite and damped or bounded
    for o in o32:
        assert torch.isfinite(torch.view_as_real(o)).all()
    b32.close()
    b64.close()
