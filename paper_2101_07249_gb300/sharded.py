"""Column-sharded randomised EVD: the sketch of Section 4 with its probe
columns partitioned over the ranks of a process group (one GPU per rank).

The paper observes that the k + l products with A in each block product are
independent and can be parallelised.  Here rank r owns the probe columns
[c_r, c_{r+1}) through every block product with A (a forward and an adjoint
sweep per column, no communication), and the block linear algebra runs on a
row partition: an all-to-all turns the column-sharded product A Z into
row blocks, every rank forms the partial Gram matrix of its rows, and one
all-reduce of the K x K FP64 matrix gives the whole Gram matrix, whose small
factorisation (Cholesky for CholeskyQR2, the symmetric EVD of Rayleigh-Ritz)
each rank repeats.  The Ritz vectors come out row-partitioned and an
all-gather gives every rank the full basis for its (replicated) PCG.

REVD(q) as the single-device sketch computes it (Alg. 3 plus q power
iterations): Z = orth(A G); q times Z = orth(A Z); K_1 = Z^T (A Z);
K_1 = W Theta W^T; U = Z W[:, :k].  orth is CholeskyQR2, the same
orthonormalisation as the single-device path.

Every numerical step is a library call (``ops``: the block Hessian product,
the Gram of a row block, the Cholesky inverse, the tall-by-small product, the
small symmetric EVD); torch.distributed moves the data.  ``LibraryOps`` binds
them to one wc4d context; the multi-process tests on the CPU bind the same
interface to the FP64 oracle.
"""
from __future__ import annotations

import numpy as np


def partition(total, parts):
    """Contiguous split of range(total) into `parts` blocks (sizes differ by at most one)."""
    base, extra = divmod(int(total), int(parts))
    edges = [0]
    for r in range(parts):
        edges.append(edges[-1] + base + (1 if r < extra else 0))
    return edges


class Comm:
    """The process group the sketch runs over (torch.distributed), or one
    process when the group is not initialised."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.size = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0

    def all_reduce(self, t):
        if self.dist:
            self.dist.all_reduce(t, group=self.group)
        return t

    def all_to_all(self, out, inp, out_splits, in_splits):
        if self.dist:
            self.dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)
        else:
            out.copy_(inp)
        return out

    def all_gather(self, parts_out, t):
        if self.dist:
            self.dist.all_gather(parts_out, t.contiguous(), group=self.group)
        else:
            parts_out[0].copy_(t)
        return parts_out


class LibraryOps:
    """The numerical steps bound to one wc4d context (device tensors).
    Blocks are torch tensors of shape (columns, rows): row i of the tensor
    is column i of the column-major block."""

    def __init__(self, ctx, precision):
        import torch
        from . import FP64, _fdtype
        self.ctx, self.precision = ctx, precision
        self.dtype = _fdtype(precision) or torch.float64
        self.device = "cuda"
        self.fp64 = FP64

    def zeros(self, *shape, dtype=None):
        import torch
        return torch.zeros(*shape, dtype=dtype or self.dtype, device=self.device)

    def hvp(self, X):                       # (m, nA) -> A X
        from . import wc4d_hvp
        Y = self.zeros(*X.shape)
        if X.shape[0]:
            wc4d_hvp(self.ctx, X.contiguous(), Y, X.shape[0], X.shape[1], self.precision)
        return Y

    def gram(self, A, B):                   # (ma, rows), (mb, rows) -> A^T B (ma, mb) FP64, column-major
        from . import wc4d_gram
        import torch
        C = self.zeros(B.shape[0], A.shape[0], dtype=torch.float64)   # (mb, ma) row-major = (ma, mb) column-major
        if A.shape[1]:
            wc4d_gram(self.ctx, A.contiguous(), A.shape[1], B.contiguous(), B.shape[1], A.shape[1], A.shape[0],
                      B.shape[0], C, self.precision)
        return C

    def chol_inverse(self, G):              # (m, m) column-major SPD -> R^{-1} column-major
        from . import wc4d_chol_inverse
        import torch
        R = self.zeros(*G.shape, dtype=torch.float64)
        wc4d_chol_inverse(self.ctx, G.shape[0], G.contiguous(), R)
        return R

    def times_small(self, Y, W, k=None):    # (m, rows) x (m, k) column-major W -> (k, rows)
        from . import wc4d_tall_times_small
        m = Y.shape[0]
        k = W.shape[0] if k is None else int(k)      # W stored (k_all, m): column j of W is row j
        Z = self.zeros(k, Y.shape[1])
        if Y.shape[1]:
            wc4d_tall_times_small(self.ctx, Y.contiguous(), Y.shape[1], Y.shape[1], m, W.contiguous(), k, Z,
                                  Y.shape[1], self.precision)
        return Z

    def symeig(self, S):                    # (m, m) column-major symmetric -> (theta decreasing, V column-major)
        from . import wc4d_symeig
        import torch
        V = self.zeros(*S.shape, dtype=torch.float64)
        w = wc4d_symeig(self.ctx, S.shape[0], S.contiguous(), V)
        return w, V

    def install(self, k, U, theta):
        from . import wc4d_set_ritz
        wc4d_set_ritz(self.ctx, int(k), U.double().contiguous(), np.asarray(theta, dtype=np.float64))


def _cols_to_rows(comm, ops, Xc, cols, rows):
    """Column partition (this rank: columns cols[r]..cols[r+1] of every row)
    -> row partition (this rank: rows rows[r]..rows[r+1] of every column)."""
    import torch
    P, r = comm.size, comm.rank
    mc, nr = cols[r + 1] - cols[r], rows[r + 1] - rows[r]
    inp = torch.cat([Xc[:, rows[s]:rows[s + 1]].reshape(-1) for s in range(P)])
    out = ops.zeros(cols[-1] * nr)
    comm.all_to_all(out, inp, [(cols[s + 1] - cols[s]) * nr for s in range(P)],
                    [mc * (rows[s + 1] - rows[s]) for s in range(P)])
    return out.reshape(cols[-1], nr)


def _rows_to_cols(comm, ops, Xr, cols, rows):
    """Row partition -> column partition (the inverse of _cols_to_rows)."""
    import torch
    P, r = comm.size, comm.rank
    nr = rows[r + 1] - rows[r]
    inp = torch.cat([Xr[cols[s]:cols[s + 1], :].reshape(-1) for s in range(P)])
    mc = cols[r + 1] - cols[r]
    out = ops.zeros(mc * rows[-1])
    comm.all_to_all(out, inp, [mc * (rows[s + 1] - rows[s]) for s in range(P)],
                    [(cols[s + 1] - cols[s]) * nr for s in range(P)])
    pieces, off = [], 0
    for s in range(P):
        ns = rows[s + 1] - rows[s]
        pieces.append(out[off:off + mc * ns].reshape(mc, ns))
        off += mc * ns
    return torch.cat(pieces, dim=1) if mc else ops.zeros(0, rows[-1])


def _orth_rows(comm, ops, Yr):
    """CholeskyQR2 of a row-partitioned block: two passes of G = sum_r Y_r^T
    Y_r (all-reduce), G = R^T R, Y_r <- Y_r R^{-1}."""
    for _ in range(2):
        G = comm.all_reduce(ops.gram(Yr, Yr))
        Rinv = ops.chol_inverse(G)
        Yr = ops.times_small(Yr, Rinv)
    return Yr


def sharded_revd(ops, comm, G_cols, k, q=1):
    """REVD(q) with the probe columns sharded over `comm`.  G_cols: this
    rank's probe columns (its slice of the K = k + l columns, shape (m_r, nA);
    the slices in rank order make up the whole block).  Returns the k Ritz
    values (decreasing, on every rank) and this rank's rows of the Ritz
    vectors ((k, n_r), rows partition(nA, size)[rank] ..)."""
    import torch
    nA = G_cols.shape[1]
    counts = torch.tensor([G_cols.shape[0]], dtype=torch.int64)
    if comm.dist:
        allc = [torch.zeros(1, dtype=torch.int64) for _ in range(comm.size)]
        comm.dist.all_gather(allc, counts.to(allc[0].device), group=comm.group)
        sizes = [int(c.item()) for c in allc]
    else:
        sizes = [int(counts.item())]
    cols = [0]
    for c in sizes:
        cols.append(cols[-1] + c)
    rows = partition(nA, comm.size)
    Y = ops.hvp(G_cols)                                         # A G (own columns)
    Z = _orth_rows(comm, ops, _cols_to_rows(comm, ops, Y, cols, rows))
    for _ in range(q):
        AZ = ops.hvp(_rows_to_cols(comm, ops, Z, cols, rows))
        Z = _orth_rows(comm, ops, _cols_to_rows(comm, ops, AZ, cols, rows))
    AZ = _cols_to_rows(comm, ops, ops.hvp(_rows_to_cols(comm, ops, Z, cols, rows)), cols, rows)
    K1 = comm.all_reduce(ops.gram(Z, AZ))                        # Z^T (A Z)
    theta, W = ops.symeig(K1)
    Ur = ops.times_small(Z, W, k)                                # this rank's rows of Z W[:, :k]
    return np.asarray(theta[:k]), Ur, rows


def gather_rows(comm, ops, Ur, rows):
    """All-gather a row-partitioned block (k, n_r) into the full (k, nA)
    (blocks padded to the largest n_r: collectives move equal sizes)."""
    import torch
    nmax = max(rows[s + 1] - rows[s] for s in range(comm.size))
    mine = ops.zeros(Ur.shape[0], nmax)
    mine[:, :Ur.shape[1]] = Ur
    parts = [ops.zeros(Ur.shape[0], nmax) for _ in range(comm.size)]
    comm.all_gather(parts, mine)
    return torch.cat([parts[s][:, :rows[s + 1] - rows[s]] for s in range(comm.size)], dim=1)
