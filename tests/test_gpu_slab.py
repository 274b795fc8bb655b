"""Slab-fused Tucker operators of 3D split-BF16 handles (Sec. 3.2, Eq. fKu_diag).

Kernel by kernel: the fused mode-1 + mode-2 product per j_3 slab and the
mode-3 product on the natural order (MN-major operand) against the FP64
kernels of the rotating layout on the same data.  Whole operators and
schemes: the slab-fused form forced on a handle against the FP64 oracle, at
the tolerances of the rotating form (test_gpu_bf16x3.py).
"""
import numpy as np
import pytest

from oracle import adjoint, schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import PARS, rand_tensor, rel, rel_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# every n_mu rounds to the same p_mu for FP64 handles (multiples of 4) and
# BF16X3 handles (multiples of 8), so both handles share the internal layout
KERNEL_SHAPES = [
    [30, 22, 134],   # p = (32, 24, 136): N2 = 32 (one output box, idle store warps), 3 ragged k-chunks in direction 3
    [134, 150, 6],   # p = (136, 152, 8): 2 i1-blocks (ragged), N2 = 160 > p2, two M2 boxes, ragged k-chunks
    [256, 256, 8],   # p = (256, 256, 8): the full 256 x 256 slab
    [302, 22, 6],    # p = (304, 24, 8): three i1-blocks (the last ragged), ten 32-wide k-chunks in stage 1
    [14, 6, 518],    # p = (16, 8, 520): N2 = 16, one partly valid output box; mode 3 with five ragged i-blocks
]
BOXES = [(-4.0, 4.0), (-3.0, 3.0), (-5.0, 5.0)]
AL = [1.3, 1.7, 1.5]
TOL_ONE = 3e-5    # one split-BF16 product (as the rotating kernel's test)
TOL_TWO = 5e-5    # two chained split-BF16 products with a re-split between them
TOL_APPLY = 1e-4
TOL_INTEGRATE = 1e-4


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def _split(x):
    """FP32 device tensor -> the split form (hi planes, then lo planes)."""
    hi = x.to(torch.bfloat16)
    lo = (x - hi.float()).to(torch.bfloat16)
    return torch.cat([hi, lo])


def _unsplit(y):
    n = y.numel() // 2
    return y[:n].float() + y[n:].float()


def _pair(fc, ns):
    s64 = fc.Solver(ns, BOXES, AL, **PARS, precision="fp64")
    s32 = fc.Solver(ns, BOXES, AL, **PARS, precision="bf16x3")
    p = [(n + 7) // 8 * 8 for n in ns]
    P = fc.fcgle_internal_elems(s32.h)
    assert P == fc.fcgle_internal_elems(s64.h) == int(np.prod(p))
    return s64, s32, p, P


@pytest.mark.parametrize("ns", KERNEL_SHAPES)
@pytest.mark.parametrize("fwd", [True, False])
def test_slab12_matches_two_fp64_products(fc, ns, fwd):
    s64, s32, p, P = _pair(fc, ns)
    gen = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float32, generator=gen)
    Xs = _split(X)
    # reference: mode 1 then mode 2 in the rotating layout, FP64, on the split value
    X64 = _unsplit(Xs).double()
    Y1 = torch.empty_like(X64)
    Y2 = torch.empty_like(X64)
    fc.fcgle_mode_product(s64.h, 0, int(fwd), X64, Y1)   # [c][i1][j3][j2]
    fc.fcgle_mode_product(s64.h, 1, int(fwd), Y1, Y2)    # [c][i2][i1][j3]
    ref = Y2.view(2, p[1], p[0], p[2]).permute(0, 3, 1, 2).contiguous().view(-1)   # [c][j3][i2][i1]
    Y = torch.empty(4 * P, device="cuda", dtype=torch.bfloat16)
    fc.fcgle_mode_product(s32.h, 0, int(fwd) | 2 | 8, Xs, Y)
    s64.sync()
    s32.sync()
    assert rel_dev(_unsplit(Y), ref) <= TOL_TWO
    s64.close()
    s32.close()


@pytest.mark.parametrize("ns", KERNEL_SHAPES)
@pytest.mark.parametrize("fwd", [True, False])
def test_natural_order_product_matches_fp64(fc, ns, fwd):
    s64, s32, p, P = _pair(fc, ns)
    R = P // p[2]
    gen = torch.Generator(device="cuda").manual_seed(8)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float32, generator=gen)
    Xs = _split(X)
    # reference: the rotating-layout FP64 product on the transposed input X[c][r][k]
    Xrot = _unsplit(Xs).double().view(2, p[2], R).transpose(1, 2).contiguous().view(-1)
    ref = torch.empty_like(Xrot)
    fc.fcgle_mode_product(s64.h, 2, int(fwd), Xrot, ref)
    Y = torch.empty(4 * P, device="cuda", dtype=torch.bfloat16)
    fc.fcgle_mode_product(s32.h, 2, int(fwd) | 2 | 16, Xs, Y)
    s64.sync()
    s32.sync()
    assert rel_dev(_unsplit(Y), ref) <= TOL_ONE
    s64.close()
    s32.close()


def test_flag_validation(fc):
    ns = [30, 22, 134]
    s = fc.Solver(ns, BOXES, AL, **PARS, precision="bf16x3")
    P = fc.fcgle_internal_elems(s.h)
    X = torch.zeros(4 * P, device="cuda", dtype=torch.bfloat16)
    Y = torch.empty_like(X)
    for direction, flags in ((0, 8), (1, 2 | 8), (0, 2 | 16), (2, 2 | 8 | 16)):
        with pytest.raises(fc.FcgleError):
            fc.fcgle_mode_product(s.h, direction, flags, X, Y)
    s.close()
    s2 = fc.Solver([40, 36], BOXES[:2], AL[:2], **PARS, precision="bf16x3")
    with pytest.raises(fc.FcgleError):
        s2.set_tucker_form("slab")
    s2.set_tucker_form("rotating")
    s2.close()
    s64 = fc.Solver(ns, BOXES, AL, **PARS, precision="fp64")
    with pytest.raises(fc.FcgleError):
        s64.set_tucker_form("slab")
    with pytest.raises(fc.FcgleError):
        s64.set_tucker_form(7)
    s64.close()
    big = fc.Solver([8, 264, 8], BOXES, AL, **PARS, precision="bf16x3")   # p_2 = 264 > 256
    with pytest.raises(fc.FcgleError):
        big.set_tucker_form("slab")
    big.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.complex64).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("ns", [[33, 20, 29], [134, 150, 6], [40, 256, 24], [302, 22, 6]])
def test_apply_f_slab_form(fc, ns):
    P = tensor.Problem(ns, BOXES, AL, *PARS.values())
    S = tensor.Spectral(P)
    s = fc.Solver(ns, BOXES, AL, **PARS, precision="bf16x3")
    s.set_tucker_form("slab")
    V = rand_tensor(ns, 30)
    v = _dev(V)
    V32 = V.astype(np.complex64).astype(np.complex128)
    for th in (1e-3, 0.07):
        for func, k in (("inv", 0), ("exp", 0), ("phi", 1), ("phi", 2), ("phi", 3), ("phi", 4)):
            got = _host(s.apply_f(func, k, th, v))
            ref = S.apply_f(func, k, th, V32)
            assert rel(got, ref) <= TOL_APPLY, (func, k, th, rel(got, ref))
    s.sync()
    s.close()


@pytest.mark.parametrize("scheme", ["lie", "lawson_euler", "lawson_rk2", "etd2rk", "krogstad", "lbdf2", "strang"])
def test_integrate_slab_form(fc, scheme):
    ns, boxes, al = [33, 20, 29], [(-4.0, 4.0), (-3.0, 3.0), (-5.0, 5.0)], [1.5, 1.2, 1.9]
    P = tensor.Problem(ns, boxes, al, *PARS.values())
    u0 = (0.8 * inputs.gaussian_pulse(ns, [(-2.0, 2.0)] * 3) * np.exp(1j * rand_tensor(ns, 4).real))
    u0 = u0.astype(np.complex64).astype(np.complex128)
    src = [] if scheme == "strang" else [0.3 * rand_tensor(ns, 5).astype(np.complex64).astype(np.complex128)]
    sig = [] if scheme == "strang" else [-0.7 + 2.0j]
    g = schemes.Nonlinearity(P, sig, src)
    tau, m = 0.013, 7
    ref = schemes.integrate(tensor.Spectral(P), g, scheme, tau, m, u0, t0=0.2)
    s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
    s.set_tucker_form("slab")
    if src:
        s.set_source(sig, [_dev(x) for x in src])
    got = _host(s.integrate(scheme, tau, m, _dev(u0), t0=0.2))
    s.sync()
    assert rel(got, ref) <= TOL_INTEGRATE, rel(got, ref)
    s.close()


def test_forms_agree_at_full_slab_size(fc):
    """256 x 256 x 24 Krogstad, 5 steps: the slab-fused and the rotating forms
    agree to the split-BF16 level, and both stay within 1e-5 of the FP64 GPU
    result (measured on GB300: 2.2e-6 max-elementwise for the rotating form)."""
    ns = [256, 256, 24]
    boxes = [(-10.0, 10.0), (-10.0, 10.0), (-3.0, 3.0)]
    al = [1.2, 1.5, 1.8]
    u0 = inputs.gaussian_random_phase(ns, boxes, seed=2)
    out = {}
    for form in ("rotating", "slab"):
        s = fc.Solver(ns, boxes, al, **PARS, precision="bf16x3")
        s.set_tucker_form(form)
        out[form] = s.integrate("krogstad", 1e-3, 5, torch.from_numpy(u0).to(torch.complex64).cuda())
        s.sync()
        s.close()
    s64 = fc.Solver(ns, boxes, al, **PARS, precision="fp64")
    ref = s64.integrate("krogstad", 1e-3, 5, torch.from_numpy(u0).cuda())
    s64.sync()
    s64.close()
    d_forms = rel_dev(out["slab"], out["rotating"].to(torch.complex128))
    d_ref = {form: rel_dev(out[form], ref) for form in out}
    print(f"slab vs rotating {d_forms:.2e}; vs FP64: {d_ref}")
    # the split-BF16 bound of the time integration (1e-5 relative at T), on the
    # larger of the norm-wise and max-elementwise errors
    assert d_forms <= 1e-5
    for form in out:
        assert d_ref[form] <= 1e-5, form


def test_adjoint_slab_form(fc):
    """The adjoint's Tucker operators in the slab-fused form: the gradient of
    Lawson-RK2 against the oracle's discrete adjoint."""
    ns, boxes, al = [12, 10, 9], [(-3.0, 3.0), (-2.5, 2.5), (-2.0, 2.0)], [1.5, 1.3, 1.7]
    pars = dict(nu=1.0, eta=0.5, gamma=0.8, kappa=1.2, zeta=0.4)
    tau, m = 0.02, 9
    P = tensor.Problem(ns, boxes, al, *pars.values())
    S = tensor.Spectral(P)
    rng = np.random.default_rng(11)
    g = schemes.Nonlinearity(P)
    u0 = inputs.gaussian_pulse(ns, [(-2.0, 2.0)] * 3) * np.exp(1j * rng.uniform(0, 1, size=P.shape))
    target = 0.9 * adjoint.forward(S, g, tau, m, u0)[0][-1] + 0.01
    J, gu, gp = adjoint.gradient(S, g, tau, m, u0, target)
    s = fc.Solver(ns, boxes, al, **pars, precision="bf16x3")
    s.set_tucker_form("slab")
    loss, g_u0, g_par = s.adjoint("lawson_rk2", tau, m, _dev(u0), _dev(target), ckpt_every=3)
    got = g_u0.cpu().numpy().astype(np.complex128)
    assert loss == pytest.approx(J, rel=2e-4)
    assert rel(got, gu) <= 2e-4
    np.testing.assert_allclose(g_par, gp, rtol=2e-4, atol=2e-4 * np.abs(gp).max())
    s.close()
