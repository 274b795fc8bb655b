"""fcgle_norm_static, the allocation-free norm (scratch in static device
memory), against the handle-based fcgle_norm on the same tensors, two calls in
a row; and its size limit.  Kept in the last test file so that it also runs
after everything else in one process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def test_rejects_tensors_beyond_the_scratch(fc):
    # 1024^3 complex entries need 131072 partial sums; the scratch holds 32768.
    # The size check comes before any CUDA call, so this needs no GPU.
    p = fc.make_params([1024, 1024, 1024], [(-1.0, 1.0)] * 3, [1.5] * 3, 1.0, 0.0, 0.0, 1.0, 0.0)
    with pytest.raises(fc.FcgleError) as e:
        fc.fcgle_norm_static(p, 1, None)
    assert e.value.status == fc.FCGLE_ERR_INVALID_ARG
    assert "at most 268435456" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("ns", [[1], [37, 5], [300, 301], [64, 65, 66], [8192, 8192 * 4]])
def test_matches_handle_norm_twice(fc, prec, ns):
    boxes = [(-10.0, 10.0 + k) for k in range(len(ns))]
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    g = torch.Generator(device="cuda").manual_seed(11 + len(ns))
    shape = tuple(reversed(ns))
    if len(ns) == 2 and ns[0] == 8192:       # exactly the largest size the scratch takes
        shape = (8192 * 4, 8192)
    u = torch.randn(shape, dtype=dt, device="cuda", generator=g)
    p = fc.make_params(list(reversed(shape)), boxes, [1.5] * len(ns), 1.0, 0.5, 1.0, 1.0, 0.5, precision=prec)
    torch.cuda.synchronize()
    got1 = fc.fcgle_norm_static(p, u)
    got2 = fc.fcgle_norm_static(p, u)
    cell = np.prod([(b - a) / (n + 1) for n, (a, b) in zip(list(reversed(shape)), boxes)])
    ref_t = float(np.sqrt(cell * float(torch.sum(torch.abs(u.to(torch.complex128)) ** 2))))
    assert got1 == got2                      # fixed chunking: bitwise reproducible
    assert abs(got1 - ref_t) <= 1e-12 * ref_t
    if int(np.prod(shape)) <= 4 * 10 ** 7 and max(shape) <= 8192 and min(shape) >= 3:
        h = fc.fcgle_setup(list(reversed(shape)), boxes, [1.5] * len(ns), 1.0, 0.5, 1.0, 1.0, 0.5, precision=prec)
        ref = fc.fcgle_norm(h, u)
        fc.fcgle_destroy(h)
        assert abs(got1 - ref) <= 1e-12 * ref
        assert abs(got2 - ref) <= 1e-12 * ref
