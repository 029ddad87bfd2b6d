"""The column-sharded sketch's numerical steps bound to the library
(sharded.LibraryOps: block Hessian products, Gram of row blocks, Cholesky
inverse, tall-by-small products, small symmetric EVD, all through the
C-ABI) in one process: the same Ritz values as the library's own REVD on the
same probes, and the new building blocks against numpy on the same data.
The multi-rank exchange is covered on the CPU (tests/test_sharded_gloo.py)."""
import numpy as np
import pytest

from paper_2101_07249_gb300 import inputs, sharded

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu


def test_building_blocks_match_numpy():
    cfg = inputs.scaled(inputs.TINY, n=64, N=3, k=6, l=2)
    S = w.Solver(cfg)
    g = np.random.default_rng(4)
    rows, ma, mb = 1000, 7, 5
    A, B = g.standard_normal((ma, rows)), g.standard_normal((mb, rows))
    C = torch.zeros(mb, ma, dtype=torch.float64, device="cuda")
    w.wc4d_gram(S.ctx, torch.as_tensor(A, device="cuda"), rows, torch.as_tensor(B, device="cuda"), rows, rows, ma, mb,
                C)
    assert np.allclose(C.cpu().numpy().T, A @ B.T, rtol=1e-13, atol=1e-12)
    C32 = torch.zeros(mb, ma, dtype=torch.float64, device="cuda")
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    w.wc4d_gram(S.ctx, torch.as_tensor(A32, device="cuda"), rows, torch.as_tensor(B32, device="cuda"), rows, rows,
                ma, mb, C32, w.MIXED)
    assert np.allclose(C32.cpu().numpy().T, A32.astype(np.float64) @ B32.astype(np.float64).T, rtol=1e-12, atol=1e-11)
    Gm = A @ A.T + np.eye(ma)
    Rinv = torch.zeros(ma, ma, dtype=torch.float64, device="cuda")
    w.wc4d_chol_inverse(S.ctx, ma, torch.as_tensor(Gm.T.copy(), device="cuda"), Rinv)
    R = np.linalg.cholesky(Gm).T
    assert np.allclose(Rinv.cpu().numpy().T, np.linalg.inv(R), rtol=1e-12, atol=1e-13)
    Wm = g.standard_normal((ma, 3))
    Z = torch.zeros(3, rows, dtype=torch.float64, device="cuda")
    w.wc4d_tall_times_small(S.ctx, torch.as_tensor(A, device="cuda"), rows, rows, ma,
                            torch.as_tensor(Wm.T.copy(), device="cuda"), 3, Z, rows)
    assert np.allclose(Z.cpu().numpy(), (A.T @ Wm).T, rtol=1e-13, atol=1e-12)
    with pytest.raises(w.WC4DError) as e:           # not positive definite
        w.wc4d_chol_inverse(S.ctx, 2, torch.as_tensor(np.array([[1.0, 2.0], [2.0, 1.0]]), device="cuda"),
                            torch.zeros(2, 2, dtype=torch.float64, device="cuda"))
    assert e.value.status == w.ENOTSPD
    S.close()


@pytest.mark.parametrize("q", [0, 1])
def test_sharded_revd_single_rank_matches_library_sketch(q):
    cfg = inputs.scaled(inputs.TINY, n=128, N=6, k=12, l=4, obs_stride=6)
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    G = inputs.probes(9, cfg.nA, cfg.K)
    th_lib = w.wc4d_sketch(S.ctx, w.REVD, cfg.k, cfg.l, q, 0, torch.as_tensor(G, device="cuda"), w.FP64)
    ops = sharded.LibraryOps(S.ctx, w.FP64)
    comm = sharded.Comm()
    theta, Ur, rows = sharded.sharded_revd(ops, comm, torch.as_tensor(G, device="cuda"), cfg.k, q=q)
    assert np.allclose(theta, th_lib, rtol=1e-10)
    U = sharded.gather_rows(comm, ops, Ur, rows)
    Uh = U.cpu().numpy()
    assert np.abs(Uh @ Uh.T - np.eye(cfg.k)).max() < 1e-12
    ops.install(cfg.k, U, theta)                       # usable as the context's LMP
    assert w.wc4d_ritz_count(S.ctx) == cfg.k
    S.close()
