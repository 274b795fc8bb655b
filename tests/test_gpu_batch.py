"""Batched instances: each instance of a batch (CUDA-graph replay or direct
enqueue over several streams) equals the same instance run alone, bit for bit,
and one instance matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import schemes, tensor
from paper_2510_21394_gb300 import inputs
from helpers import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _specs(seed=2, n2=4, n3=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for d, cnt, lo, hi in ((2, n2, 20, 90), (3, n3, 8, 30)):
        for _ in range(cnt):
            n = int(rng.integers(lo, hi + 1))
            out.append(dict(ns=[n] * d, boxes=[(-10.0, 10.0)] * d, alphas=list(rng.uniform(1.1, 1.9, d)),
                            nu=float(rng.uniform(0.5, 2)), eta=float(rng.uniform(-1, 1)),
                            gamma=float(rng.uniform(0, 1)), kappa=float(rng.uniform(0.5, 2)),
                            zeta=float(rng.uniform(-1, 1))))
    return out


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
@pytest.mark.parametrize("scheme", ["etd2rk", "lbdf2", "krogstad"])
@pytest.mark.parametrize("graph", [True, False, "grouped"])
def test_batch_equals_single_runs(fc, prec, scheme, graph):
    specs = _specs()
    dt = torch.complex64 if prec == "bf16x3" else torch.complex128
    b = fc.Batch(specs, precision=prec, nstreams=3)
    u0 = [torch.from_numpy(inputs.gaussian_pulse(sp["ns"], [(-3.0, 3.0)] * len(sp["ns"]))).to(dt).cuda()
          for sp in specs]
    tau, m = 5e-3, 6
    grouped = graph == "grouped"
    use_graph = bool(graph)
    k0, _ = b.launches()
    outs = b.integrate(scheme, tau, m, u0, use_graph=use_graph, grouped=grouped)
    outs2 = b.integrate(scheme, tau, m, u0, use_graph=use_graph, grouped=grouped)   # cached plan, same result
    torch.cuda.synchronize()
    k, gl = b.launches()
    assert k > 0 and (gl > 0) == use_graph
    if grouped and prec == "bf16x3":
        # grouped: a step of all 7 instances is a few launches (3 per Tucker operator of
        # this 2D + 3D mix), not one per instance and mode product
        steps = 2 * (m - (1 if scheme == "lbdf2" else 0))
        assert gl == steps
    for sp, u, o, o2 in zip(specs, u0, outs, outs2):
        s = fc.Solver(sp["ns"], sp["boxes"], sp["alphas"], sp["nu"], sp["eta"], sp["gamma"], sp["kappa"],
                      sp["zeta"], precision=prec)
        # a batch runs every Tucker operator in the rotating form; a single
        # handle may run the slab-fused form (autotuned), which rounds differently
        s.set_tucker_form("rotating")
        ref = s.integrate(scheme, tau, m, u)
        torch.cuda.synchronize()
        assert torch.equal(o, ref) and torch.equal(o2, ref)
        s.close()
    b.close()


def test_batch_instance_against_oracle(fc):
    specs = _specs(seed=5, n2=2, n3=2)
    b = fc.Batch(specs, precision="bf16x3")
    u0n = [inputs.gaussian_pulse(sp["ns"], [(-3.0, 3.0)] * len(sp["ns"])) for sp in specs]
    u0 = [torch.from_numpy(x).to(torch.complex64).cuda() for x in u0n]
    outs = b.integrate("etd2rk", 5e-3, 8, u0)
    torch.cuda.synchronize()
    for sp, x0, o in zip(specs, u0n, outs):
        P = tensor.Problem(sp["ns"], sp["boxes"], sp["alphas"], sp["nu"], sp["eta"], sp["gamma"], sp["kappa"],
                           sp["zeta"])
        ref = schemes.integrate(tensor.Spectral(P), schemes.Nonlinearity(P), "etd2rk", 5e-3, 8,
                                x0.astype(np.complex64).astype(np.complex128))
        got = o.cpu().numpy().astype(np.complex128)
        assert rel(got, ref) <= 1e-4
    b.close()


def test_batch_with_source_falls_back_to_direct_launches(fc):
    specs = _specs(seed=7, n2=2, n3=1)
    b = fc.Batch(specs, precision="bf16x3")
    sp = specs[0]
    h = b.instance(0)
    S = torch.ones(tuple(reversed(sp["ns"])), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()               # set_source runs on the instance's internal stream
    fc.fcgle_set_source(h, [-1.0], [S])
    u0 = [torch.zeros(tuple(reversed(x["ns"])), dtype=torch.complex64, device="cuda") for x in specs]
    outs = b.integrate("etd2rk", 1e-2, 3, u0, use_graph=True)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        fc.fcgle_sync(b.instance(i))       # no bounded device wait gave up
    assert b.launches()[1] == 0            # no graph: the source makes the steps time dependent
    assert float(torch.abs(outs[0]).max()) > 0 and float(torch.abs(outs[1]).max()) == 0
    b.close()


@pytest.mark.parametrize("graph", [True, "grouped"])
def test_batch_replays_new_coefficients(fc, graph):
    """A captured step holds the coefficients it was built with: after
    fcgle_set_coefficients on one instance the batch must rebuild it, and the
    result must equal that of a fresh batch created with the new values."""
    specs = _specs(seed=7, n2=3, n3=2)
    dt = torch.complex64
    u0 = [torch.from_numpy(inputs.gaussian_pulse(sp["ns"], sp["boxes"])).to(dt).cuda() for sp in specs]
    grouped = graph == "grouped"
    b = fc.Batch(specs, precision="bf16x3")
    b.integrate("etd2rk", 1e-3, 4, u0, use_graph=True, grouped=grouped)
    sp1 = dict(specs[1])
    sp1["gamma"] = sp1["gamma"] + 0.7
    sp1["zeta"] = -sp1["zeta"]
    fc.fcgle_set_coefficients(b.instance(1), sp1["nu"], sp1["eta"], sp1["gamma"], sp1["kappa"], sp1["zeta"])
    got = b.integrate("etd2rk", 1e-3, 4, u0, use_graph=True, grouped=grouped)
    specs2 = list(specs)
    specs2[1] = sp1
    b2 = fc.Batch(specs2, precision="bf16x3")
    ref = b2.integrate("etd2rk", 1e-3, 4, u0, use_graph=True, grouped=grouped)
    torch.cuda.synchronize()
    for i in range(len(specs)):
        fc.fcgle_sync(b.instance(i))
        assert torch.equal(got[i], ref[i]), i
    b.close()
    b2.close()
