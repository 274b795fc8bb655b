"""Partitioning across ranks (host logic, CPU): the greedy instance
assignment of the batched workload, and the slab decomposition of one
instance, whose Tucker operators (Eq. fKu_diag) run on gloo ranks with the
oracle's mode products and one all-to-all each, against the single-process
oracle f(theta K) v."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2510_21394_gb300 import inputs, sharding  # noqa: E402


def test_assignment_covers_every_instance_once_and_balances():
    sizes = [sp["ns"] for sp in inputs.batched_instances()]
    cost = [sharding.instance_cost(ns) for ns in sizes]
    for world in (1, 2, 3, 4, 8):
        owner, load = sharding.assign_instances(sizes, world)
        assert sorted(i for r in range(world) for i in sharding.instances_of(owner, r)) == list(range(len(sizes)))
        for r in range(world):
            assert load[r] == pytest.approx(sum(c for c, o in zip(cost, owner) if o == r))
        # greedy longest-processing-time bound: no rank exceeds the lightest by more than one instance
        assert max(load) - min(load) <= max(cost) + 1e-6 * max(load)
        assert sharding.assign_instances(sizes, world) == (owner, load)   # every rank computes the same
    # two ranks split the 96-instance batch within 1 % of each other
    _, load = sharding.assign_instances(sizes, 2)
    assert max(load) / min(load) < 1.01


def test_block_ranges_tile_the_index():
    for n in (1, 5, 7, 256, 1023):
        for world in (1, 2, 3, 8):
            rs = [sharding.block_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sz = [hi - lo for lo, hi in rs]
            assert max(sz) - min(sz) <= 1


def _slab_worker(rank, world, port, ns, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import tensor
    from paper_2510_21394_gb300 import sharding as sh
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        boxes = [(-2.0, 2.0), (-1.0, 3.0), (-1.5, 1.5)][: len(ns)]
        al = [1.2, 1.8, 1.5][: len(ns)]
        P = tensor.Problem(ns, boxes, al, 1.0, 0.6, 0.5, 1.0, -0.3)
        S = tensor.Spectral(P)
        rng = np.random.default_rng(3)
        shape = tuple(reversed(ns))
        V = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        part = sh.SlabPartition(ns, world, rank)

        def mp(X, M, mu):   # the oracle's mode product on a local block
            return torch.from_numpy(np.ascontiguousarray(tensor.mode_product(X.numpy(), M, mu)))
        Qt = [Q.T.copy() for Q in S.Q]
        out = {}
        for kind, ell, th in (("phi", 1, 0.05), ("inv", 0, 0.1), ("exp", 0, 0.03)):
            Xr = torch.from_numpy(np.ascontiguousarray(part.scatter_rows(V)))
            Xc = part.tucker_forward(Xr, Qt, mp, dist)                    # column layout
            F = torch.from_numpy(np.ascontiguousarray(part.scatter_cols(S.F(kind, ell, th))))
            Yr = part.tucker_backward(F * Xc, S.Q, mp, dist)              # row layout
            ref = part.scatter_rows(S.apply_f(kind, ell, th, V))
            out[kind] = float(np.max(np.abs(Yr.numpy() - ref)) / np.max(np.abs(ref)))
        # the two exchanges are inverse to each other
        Xr = torch.from_numpy(np.ascontiguousarray(part.scatter_rows(V)))
        back = part.to_rows(part.to_cols(Xr, dist), dist)
        out["roundtrip_exact"] = bool(torch.equal(back, Xr))
        cols = part.to_cols(Xr, dist)
        out["cols_exact"] = bool(np.array_equal(cols.numpy(), part.scatter_cols(V)))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("ns,world", [([7, 9], 2), ([5, 6, 8], 2), ([5, 6, 8], 3), ([9, 4, 7], 4)])
def test_slab_tucker_on_gloo_ranks_matches_oracle(ns, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, ns, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(world):
        o = res[r]
        assert o["roundtrip_exact"] and o["cols_exact"], (r, o)
        for kind in ("phi", "inv", "exp"):
            assert o[kind] <= 1e-13, (r, kind, o[kind])
