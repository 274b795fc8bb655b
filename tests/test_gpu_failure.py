"""Failure detection without a GPU fault.  Every mbarrier wait of the
tensor-core kernels is bounded: on expiry the kernel records a code in the
device error word and returns, the host reports FCGLE_ERR_TIMEOUT, and the
context stays usable.  The self-test runs that same wait on an mbarrier that
nothing completes (no fault, trap or endless loop: only the wait's own limit
ends it), then the tensor-core path runs a normal integration."""
import time

import numpy as np
import pytest

from helpers import PARS
from paper_2510_21394_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    return fcgle


def test_bounded_wait_gives_up_reports_and_context_survives(fc):
    t0 = time.perf_counter()
    status, code = fc.fcgle_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert status == fc.FCGLE_ERR_TIMEOUT, fc.fcgle_last_error()
    assert code == 99
    assert "code 99" in fc.fcgle_last_error()
    assert 1.9 <= dt < 60.0   # the limit is 2 s of device wall clock
    ns, boxes = [24, 20, 16], [(-2.0, 2.0)] * 3
    s = fc.Solver(ns, boxes, [1.3, 1.5, 1.7], **PARS, precision="bf16x3")
    u0 = torch.from_numpy(inputs.gaussian_pulse(ns, boxes)).to(torch.complex64).cuda()
    out = s.integrate("krogstad", 1e-3, 3, u0)
    s.sync()
    assert torch.isfinite(torch.view_as_real(out)).all()
    assert float(torch.linalg.vector_norm(out)) > 0.5 * float(torch.linalg.vector_norm(u0))
    s.close()
