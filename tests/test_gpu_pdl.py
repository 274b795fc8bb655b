"""Programmatic dependent launch changes when a mode-product kernel may start,
not what it computes: a Krogstad integration on one handle and a grouped batch
integration give bitwise the same results with FCGLE_PDL=0 (plain launches)
as with the default (dependent launches).  The library reads the switch once
per process, so each setting runs in an interpreter of its own."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2510_21394_gb300 import fcgle, inputs

ns, boxes = [72, 64, 48], [(-6.0, 6.0)] * 3
u0 = inputs.gaussian_random_phase(ns, boxes, seed=3)
s = fcgle.Solver(ns, boxes, [1.3, 1.5, 1.7], nu=1.0, eta=0.5, gamma=1.0, kappa=1.0, zeta=0.5,
                 precision="bf16x3")
a = s.integrate("krogstad", 1e-3, 12, torch.from_numpy(u0).to(torch.complex64).cuda())
specs = inputs.batched_instances()[:6]
b = fcgle.Batch(specs, precision="bf16x3")
ub = [torch.from_numpy(inputs.gaussian_pulse(sp["ns"], sp["boxes"])).to(torch.complex64).cuda() for sp in specs]
ob = b.integrate("etd2rk", 1e-3, 5, ub, grouped=True)
torch.cuda.synchronize()
np.savez(sys.argv[2], a.cpu().numpy(), *[o.cpu().numpy() for o in ob])
s.close()
b.close()
"""


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()


def _run(tmp_path, pdl):
    env = dict(os.environ)
    if pdl is None:
        env.pop("FCGLE_PDL", None)
    else:
        env["FCGLE_PDL"] = pdl
    out = str(tmp_path / ("pdl_%s.npz" % pdl))
    subprocess.run([sys.executable, "-c", RUN, ROOT, out], env=env, check=True, timeout=600)
    with np.load(out) as z:
        return [z[k] for k in sorted(z.files, key=lambda f: int(f.split("_")[1]))]


def test_pdl_bitwise_same(built, tmp_path):
    on = _run(tmp_path, None)
    off = _run(tmp_path, "0")
    assert len(on) == len(off) == 7
    for x, y in zip(on, off):
        assert x.shape == y.shape
        assert np.isfinite(x).all()
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
