"""Work partitioning across GPUs (host logic only; no arithmetic of the method).

Two ways the hot path spreads over ranks (one process per GPU):

* Independent instances (the batched workload): every instance is advanced on
  exactly one rank, with no exchange on the data path.  ``assign_instances``
  balances the ranks greedily by the mode-product work of one step, which for
  a d-dimensional instance is proportional to N * sum_mu n_mu (a mode product
  of direction mu costs 4 n_mu N real flops, Sec. 3.2), largest first onto the
  least-loaded rank (longest-processing-time order).

* One large instance: slab decomposition along the slowest index j_d.  A
  Tucker operator (Eq. fKu_diag) is a chain of mode products; modes
  1 .. d-1 never mix different j_d, so they run on each rank's slab with no
  communication.  Mode d contracts j_d, so before it the tensor is
  redistributed with one all-to-all into a layout where every rank holds all
  of j_d for a block of j_{d-1} (the "column" layout), the pencil-transpose
  pattern.  Because mode products of different directions commute, the next
  Tucker operator starts with mode d in the column layout and transposes back
  before modes d-1 .. 1, so each Tucker operator costs exactly one
  all-to-all.  Pointwise work (the spectral scalars, the nonlinearity) is
  local in either layout.

``SlabPartition`` holds the two layouts of one instance on one rank and the
exchange between them (``torch.distributed.all_to_all_single``, which NCCL and
gloo both provide); the mode products themselves are a callable supplied by
the caller, so the partition logic is independent of where they run.
"""
import numpy as np


# ------------------------------------------------------------- instances
def instance_cost(ns):
    """Mode-product work of one step of an instance with grid sizes ns (up to a
    constant factor): N * sum_mu n_mu."""
    return float(np.prod([int(n) for n in ns])) * float(sum(int(n) for n in ns))


def assign_instances(sizes, world):
    """Greedy balance of independent instances over `world` ranks.

    sizes: list of grid-size lists.  Returns (owner, load): owner[i] is the rank
    of instance i; load[r] the summed cost of rank r.  Instances are placed in
    decreasing cost (ties by index) onto the currently least-loaded rank (ties
    by the lowest rank), so the result is deterministic and every rank computes
    the same assignment without communication."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = [instance_cost(ns) for ns in sizes]
    order = sorted(range(len(sizes)), key=lambda i: (-cost[i], i))
    load = [0.0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += cost[i]
    return owner, load


def instances_of(owner, rank):
    """Indices of the instances assigned to `rank`, in increasing order."""
    return [i for i, r in enumerate(owner) if r == rank]


# ---------------------------------------------------------- one instance
def block_range(n, world, rank):
    """Contiguous block [lo, hi) of rank `rank` when n items are split into
    `world` blocks whose sizes differ by at most one (larger blocks first)."""
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


class SlabPartition:
    """The two layouts of one d-dimensional instance (d >= 2) on one rank.

    Tensors are arrays of shape (n_d, ..., n_1) (vec order, j_1 fastest).
    Row layout: this rank holds j_d in block_range(n_d) and every other index
    (shape (m_r, n_{d-1}, .., n_1)).  Column layout: this rank holds every j_d
    and j_{d-1} in block_range(n_{d-1}) (shape (n_d, k_r, n_{d-2}, .., n_1)).
    """

    def __init__(self, ns, world, rank):
        self.ns = [int(n) for n in ns]
        self.d = len(self.ns)
        if self.d < 2:
            raise ValueError("a slab decomposition needs d >= 2")
        self.world, self.rank = int(world), int(rank)
        shape = list(reversed(self.ns))            # (n_d, .., n_1)
        self.shape = shape
        self.rows = [block_range(shape[0], world, r) for r in range(world)]
        self.cols = [block_range(shape[1], world, r) for r in range(world)]
        self.inner = int(np.prod(shape[2:])) if self.d > 2 else 1   # entries per j_{d-1}

    def row_shape(self, rank=None):
        r = self.rank if rank is None else rank
        lo, hi = self.rows[r]
        return [hi - lo] + self.shape[1:]

    def col_shape(self, rank=None):
        r = self.rank if rank is None else rank
        lo, hi = self.cols[r]
        return [self.shape[0], hi - lo] + self.shape[2:]

    def scatter_rows(self, X):
        """This rank's row block of a full tensor X."""
        lo, hi = self.rows[self.rank]
        return X[lo:hi]

    def scatter_cols(self, X):
        lo, hi = self.cols[self.rank]
        return X[:, lo:hi]

    # ----------------------------------------------------------- exchange
    @staticmethod
    def _exchange(comm, send, recv_sizes):
        """all_to_all_single of the per-destination blocks `send` (flat tensors);
        complex data travel as their real views."""
        import torch
        send_sizes = [int(t.numel()) for t in send]
        sendbuf = torch.cat(send)
        recvbuf = torch.empty(sum(recv_sizes), dtype=sendbuf.dtype, device=sendbuf.device)
        if sendbuf.is_complex():
            comm.all_to_all_single(torch.view_as_real(recvbuf).reshape(-1), torch.view_as_real(sendbuf).reshape(-1),
                                   [2 * n for n in recv_sizes], [2 * n for n in send_sizes])
        else:
            comm.all_to_all_single(recvbuf, sendbuf, recv_sizes, send_sizes)
        return recvbuf

    def to_cols(self, Xr, comm):
        """Row layout -> column layout: one all-to-all.  Xr: torch tensor of
        row_shape(); returns a tensor of col_shape() (same dtype and device)."""
        import torch
        send = [Xr[:, lo:hi].reshape(-1) for lo, hi in self.cols]      # block for rank s
        tail = self.col_shape()[1:]
        recv_sizes = [(hi - lo) * int(np.prod(tail)) for lo, hi in self.rows]
        recvbuf = self._exchange(comm, send, recv_sizes)
        parts = []
        off = 0
        for (lo, hi), n in zip(self.rows, recv_sizes):
            parts.append(recvbuf[off:off + n].reshape([hi - lo] + tail))
            off += n
        return torch.cat(parts, dim=0)

    def to_rows(self, Xc, comm):
        """Column layout -> row layout: the inverse all-to-all."""
        import torch
        send = [Xc[lo:hi].reshape(-1) for lo, hi in self.rows]        # rows of rank s
        m = self.rows[self.rank][1] - self.rows[self.rank][0]
        recv_sizes = [m * (hi - lo) * self.inner for lo, hi in self.cols]
        recvbuf = self._exchange(comm, send, recv_sizes)
        parts = []
        off = 0
        for (lo, hi), n in zip(self.cols, recv_sizes):
            parts.append(recvbuf[off:off + n].reshape([m, hi - lo] + self.shape[2:]))
            off += n
        return torch.cat(parts, dim=1)

    # ------------------------------------------------------ Tucker operators
    def tucker_forward(self, Xr, mats, mode_product, comm):
        """X x_1 M_1 ... x_d M_d from the row layout; the result is in the column
        layout.  mode_product(X, M, mu) applies M along direction mu of a local
        block whose axes are (j_d, .., j_1) in order (axis d - mu)."""
        for mu in range(1, self.d):
            Xr = mode_product(Xr, mats[mu - 1], mu)
        Xc = self.to_cols(Xr, comm)
        return mode_product(Xc, mats[self.d - 1], self.d)

    def tucker_backward(self, Xc, mats, mode_product, comm):
        """The same product from the column layout, directions in the order
        d, d-1, .., 1 (mode products of different directions commute); the
        result is in the row layout."""
        Xc = mode_product(Xc, mats[self.d - 1], self.d)
        Xr = self.to_rows(Xc, comm)
        for mu in range(self.d - 1, 0, -1):
            Xr = mode_product(Xr, mats[mu - 1], mu)
        return Xr
