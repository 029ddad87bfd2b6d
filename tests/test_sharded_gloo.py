"""The column-sharded sketch (paper_2101_07249_gb300.sharded) on two and
three CPU processes over gloo: probe columns partitioned over the ranks, the
block products per rank, all-to-all to row blocks, one all-reduce of the
K x K Gram per CholeskyQR pass and of Z^T (A Z), the small problems
repeated on every rank.  The numerical steps are bound to the FP64 oracle
(on the GPU they are library calls); the Ritz values must equal the
single-process oracle REVD's on the same probes to 1e-12, and the gathered
Ritz vectors span the same subspace (through the LMP they define)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2101_07249_gb300 import inputs, sharded
from problems import oracle_problem

CFG = inputs.scaled(inputs.TINY, n=64, N=4, k=10, l=6, obs_stride=4)


class OracleOps:
    """The sketch's numerical steps on the CPU in FP64 (oracle Hessian
    product, numpy for the small dense pieces), with the layouts of
    sharded.LibraryOps: a block is a (columns, rows) tensor."""

    def __init__(self, p):
        self.p = p
        self.hvps = 0

    def zeros(self, *shape, dtype=None):
        return torch.zeros(*shape, dtype=torch.float64)

    def hvp(self, X):
        self.hvps += 1
        return torch.as_tensor(oracle.hvp(self.p, X.numpy())) if X.shape[0] else self.zeros(*X.shape)

    def gram(self, A, B):            # (mb, ma) tensor = A^T B column-major
        return torch.as_tensor((A.numpy() @ B.numpy().T).T.copy())

    def chol_inverse(self, G):
        Gm = G.numpy().T             # column-major -> matrix
        R = np.linalg.cholesky(Gm).T
        return torch.as_tensor(np.linalg.inv(R).T.copy())

    def times_small(self, Y, W, k=None):
        Wm = W.numpy().T             # m x k_all
        k = Wm.shape[1] if k is None else k
        return torch.as_tensor((Y.numpy().T @ Wm[:, :k]).T.copy())

    def symeig(self, S):
        w, V = np.linalg.eigh(0.5 * (S.numpy() + S.numpy().T))
        o = np.argsort(w)[::-1]
        return w[o], torch.as_tensor(V[:, o].T.copy())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q, out_dir):
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tw = inputs.twin(CFG)
        p = oracle_problem(CFG, xb=tw.xb)
        G = inputs.probes(3, CFG.nA, CFG.K)
        cols = sharded.partition(CFG.K, world)
        ops = OracleOps(p)
        comm = sharded.Comm()
        theta, Ur, rows = sharded.sharded_revd(ops, comm, torch.as_tensor(G[cols[rank]:cols[rank + 1]]), CFG.k, q=q)
        U = sharded.gather_rows(comm, ops, Ur, rows)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), theta=theta, U=U.numpy(), hvps=ops.hvps,
                 mycols=cols[rank + 1] - cols[rank])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,q", [(2, 1), (3, 0)])
def test_sharded_revd_matches_single_process(world, q, tmp_path):
    mp.spawn(_worker, args=(world, _free_port(), q, str(tmp_path)), nprocs=world, join=True)
    tw = inputs.twin(CFG)
    p = oracle_problem(CFG, xb=tw.xb)
    G = inputs.probes(3, CFG.nA, CFG.K)
    Uo, tho = oracle.revd(p, CFG.k, G, q=q)
    res = [np.load(tmp_path / f"r{r}.npz") for r in range(world)]
    for r in res:
        assert np.allclose(r["theta"], tho, rtol=1e-12, atol=0)
        assert int(r["hvps"]) == q + 2                       # Table 1: 2 + q block products per rank
        assert np.array_equal(r["U"], res[0]["U"])           # every rank holds the same gathered basis
    U = res[0]["U"]
    assert np.abs(U @ U.T - np.eye(CFG.k)).max() < 1e-12
    # same Ritz pairs as the oracle through the LMP they define (sign-invariant)
    c = 1.0 - 1.0 / np.sqrt(tho)
    v = inputs.block(5, CFG.nA, 3)
    Cg = v - ((v @ U.T) * c) @ U
    Co = v - ((v @ Uo.T) * c) @ Uo
    assert np.abs(Cg - Co).max() < 1e-9 * np.abs(v).max()
