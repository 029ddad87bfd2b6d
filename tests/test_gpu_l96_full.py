"""The Lorenz-96 window at its own grid size (n = 8192, the benchmark's
nonlinear window, here with N = 2 subwindows of 8 RK4 steps) against the
FP64 oracle's tangent-linear / adjoint Hessian product along the same
trajectory: one column (the PCG matvec: in FP64 one 8-CTA cluster per column
with halos in distributed shared memory, in FP32 the register-blocked sweep
with one column per CTA), a ragged block and the 256-column sketch block (two
columns per CTA in FP32), in FP64 (1e-12) and in the mixed precision (FP32
sweeps along the FP32 trajectory, 2e-5)."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

CFG = inputs.L96.replace(name="l96_n8192_N2", N=2)
_cache = {}


def setup():
    if "s" not in _cache:
        tw = inputs.twin(CFG, spinup=5.0)
        S = w.Solver(CFG, tw)
        p = oracle_problem(CFG, xb=tw.xb)
        _cache["s"] = (S, p, tw)
    return _cache["s"]


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


@pytest.mark.parametrize("K", [1, 7, 65, 256])
def test_l96_n8192_hvp_matches_oracle(K):
    S, p, _ = setup()
    nA = CFG.nA
    X = inputs.block(800 + K, nA, K)
    ref = oracle.hvp(p, X)
    Y = torch.zeros(K, nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y, K, nA, w.FP64)
    assert colrel(Y.cpu().numpy(), ref) < 1e-12
    Y32 = torch.zeros(K, nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, K, nA, w.MIXED)
    assert colrel(Y32.double().cpu().numpy(), ref) < 2e-5


def test_l96_n8192_rhs_and_sweeps_match_oracle():
    S, p, tw = setup()
    nA = CFG.nA
    r = torch.zeros(nA, dtype=torch.float64, device="cuda")
    w.wc4d_get_rhs(S.ctx, r)
    ref = oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))
    assert np.linalg.norm(r.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-12
    X = inputs.block(901, nA, 3)
    W = torch.as_tensor(X, device="cuda").clone()
    w.wc4d_apply_linv(S.ctx, W, 3, nA)
    assert colrel(W.cpu().numpy(), oracle.Linv(p, X)) < 1e-12
    W = torch.as_tensor(X, device="cuda").clone()
    w.wc4d_apply_linvT(S.ctx, W, 3, nA)
    assert colrel(W.cpu().numpy(), oracle.LinvT(p, X)) < 1e-12


@pytest.mark.parametrize("n,N,K", [(256, 3, 1), (256, 3, 70), (768, 2, 65), (2048, 2, 3), (2048, 2, 96)])
def test_l96_register_blocked_sizes_match_oracle(n, N, K):
    """Grid sizes where the FP32 register-blocked sweeps run (8 points per
    thread; n = 256: one warp, every halo wraps within it; n = 768: three
    warps; n = 2048: eight), one or two columns per CTA (K >= 64) and a
    partly filled last CTA; the FP64 products run the cluster (K <= 32) and
    one-CTA-per-column sweeps on the same grids."""
    cfg = inputs.L96.replace(name=f"l96_n{n}_N{N}", n=n, N=N, steps=4)
    tw = inputs.twin(cfg, spinup=5.0)
    S = w.Solver(cfg, tw)
    p = oracle_problem(cfg, xb=tw.xb)
    X = inputs.block(1000 + n + K, cfg.nA, K)
    ref = oracle.hvp(p, X)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y, K, cfg.nA, w.FP64)
    assert colrel(Y.cpu().numpy(), ref) < 1e-12
    Y32 = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, K, cfg.nA, w.MIXED)
    assert colrel(Y32.double().cpu().numpy(), ref) < 2e-5
    S.close()


def test_l96_fp32_sweeps_with_any_leading_dimension():
    """At subwindow boundaries the FP32 register-blocked sweeps read and write
    a thread's eight points of W with two 16-byte accesses when W and its
    leading dimension allow (ld = nA here), else with eight 4-byte ones
    (ld = nA + 1): both forms give the same L^{-1} and L^{-T}, bit for bit,
    and match the oracle's to FP32 accuracy, for one column and a block of
    two columns per CTA."""
    cfg = inputs.L96.replace(name="l96_n256_N3", n=256, N=3, steps=4)
    tw = inputs.twin(cfg, spinup=5.0)
    S = w.Solver(cfg, tw)
    p = oracle_problem(cfg, xb=tw.xb)
    nA = cfg.nA
    for K in (1, 66):
        X = inputs.block(1300 + K, nA, K)
        for apply, ref in ((w.wc4d_apply_linv, oracle.Linv(p, X)), (w.wc4d_apply_linvT, oracle.LinvT(p, X))):
            out = []
            for ld in (nA, nA + 1):
                Wb = torch.zeros(K, ld, dtype=torch.float32, device="cuda")
                Wb[:, :nA] = torch.as_tensor(X, dtype=torch.float32, device="cuda")
                apply(S.ctx, Wb, K, ld, w.MIXED)
                out.append(Wb[:, :nA].cpu())
            assert torch.equal(out[0], out[1])
            assert colrel(out[0].double().numpy(), ref) < 2e-5
    S.close()
