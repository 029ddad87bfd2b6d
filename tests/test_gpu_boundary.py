"""Boundary calls of the problem statement beyond the correlation-function
covariances: a covariance block given by its square root (circulant first
row, dense n x n matrix, scalar), an externally supplied Lorenz-96
linearisation trajectory, and externally supplied innovations -- each
against the FP64 oracle on the same operator."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu


def _circ(row):
    n = len(row)
    idx = (np.arange(n)[None, :] - np.arange(n)[:, None]) % n
    return row[idx]


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


@pytest.mark.parametrize("n", [100, 128])          # direct circulant and FFT path
@pytest.mark.parametrize("form", ["row", "dense", "mixed"])
def test_cov_sqrt_forms_match_oracle(n, form):
    """B^{1/2} and Q^{1/2} given as circulant rows, as dense matrices, or one
    of each: the Hessian product (FP64 and mixed) equals the oracle's with
    the same square roots."""
    cfg = inputs.scaled(inputs.TINY, n=n, N=4, k=6, l=2, obs_stride=5)
    tw = inputs.twin(cfg)
    S = w.Solver(cfg)
    p = oracle_problem(cfg, xb=tw.xb)
    rows = {0: p.Bsqrt, 1: p.Qsqrt}
    for b in (0, 1):
        if form == "row" or (form == "mixed" and b == 0):
            w.wc4d_set_cov_sqrt(S.ctx, b, w.COV_SQRT_CIRCULANT, rows[b])
        else:
            w.wc4d_set_cov_sqrt(S.ctx, b, w.COV_SQRT_DENSE, torch.as_tensor(_circ(rows[b]), device="cuda"))
    w.wc4d_set_background_obs(S.ctx, tw.xb, tw.y)
    X = inputs.block(70 + n, cfg.nA, 5)
    Y = torch.zeros(5, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y, 5, cfg.nA, w.FP64)
    ref = oracle.hvp(p, X)
    assert colrel(Y.cpu().numpy(), ref) < 1e-12
    Y32 = torch.zeros(5, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, 5, cfg.nA, w.MIXED)
    assert colrel(Y32.double().cpu().numpy(), ref) < 2e-5
    r = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_get_rhs(S.ctx, r)
    assert np.linalg.norm(r.cpu().numpy() - oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))) \
        <= 1e-12 * np.linalg.norm(r.cpu().numpy())
    S.close()


def test_scalar_cov_sqrt_matches_identity_covariance():
    cfg = inputs.scaled(inputs.TINY, n=128, N=3, k=6, l=2, obs_stride=4, q_kind=inputs.DIAG, q_var=0.04, q_L=1.0)
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    X = inputs.block(3, cfg.nA, 4)
    Y0 = torch.zeros(4, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y0, 4, cfg.nA, w.FP64)
    w.wc4d_set_cov_sqrt(S.ctx, 1, w.COV_SQRT_SCALAR, 0.2)           # Q = 0.2^2 I, the same block
    Y1 = torch.zeros_like(Y0)
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y1, 4, cfg.nA, w.FP64)
    p = oracle_problem(cfg, xb=tw.xb)
    assert colrel(Y1.cpu().numpy(), oracle.hvp(p, X)) < 1e-12
    assert colrel(Y1.cpu().numpy(), Y0.cpu().numpy()) < 1e-14
    with pytest.raises(w.WC4DError):
        w.wc4d_set_cov_sqrt(S.ctx, 1, w.COV_SQRT_SCALAR, -1.0)
    S.close()


def test_external_trajectory_and_innovation_match_oracle():
    """A Lorenz-96 context whose linearisation trajectory and innovations
    come from the caller (here a perturbed background's oracle run and the
    oracle's innovations): Hessian products and the right-hand side equal
    the oracle's on that trajectory."""
    cfg = inputs.L96.replace(name="l96_n256_N3", n=256, N=3, steps=4)
    tw = inputs.twin(cfg, spinup=5.0)
    xb = tw.xb + 0.1 * np.sin(np.arange(cfg.n))
    traj = oracle.l96_run(xb, cfg.F, cfg.dt, cfg.N * cfg.steps)
    S = w.Solver(cfg)
    w.wc4d_set_trajectory(S.ctx, torch.as_tensor(traj, device="cuda"))
    p = oracle_problem(cfg, xb=xb)
    d = oracle.innovation(p, xb, tw.y)
    Dm12b = 0.01 * inputs.block(7, cfg.nA, 1)[0]
    w.wc4d_set_innovation(S.ctx, torch.as_tensor(d, device="cuda"), torch.as_tensor(Dm12b, device="cuda"))
    r = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_get_rhs(S.ctx, r)
    ref = oracle.rhs(p, d, Dm12b)
    assert np.linalg.norm(r.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    for K in (1, 70):
        X = inputs.block(20 + K, cfg.nA, K)
        Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
        w.wc4d_hvp(S.ctx, torch.as_tensor(X, device="cuda"), Y, K, cfg.nA, w.FP64)
        assert colrel(Y.cpu().numpy(), oracle.hvp(p, X)) < 1e-12
        Y32 = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
        w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, K, cfg.nA, w.MIXED)
        assert colrel(Y32.double().cpu().numpy(), oracle.hvp(p, X)) < 2e-5
    # the PCG runs on the supplied operator and right-hand side
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, rel, _, _ = w.wc4d_pcg(S.ctx, x, 1e-8, 5000, 0, 0, w.FP64)
    res = ref - oracle.hvp(p, x.cpu().numpy()[None, :])[0]
    assert np.linalg.norm(res) <= 1.01e-8 * np.linalg.norm(ref)
    with pytest.raises(w.WC4DError):
        dense = w.Solver(inputs.TINY)
        try:
            w.wc4d_set_trajectory(dense.ctx, torch.zeros((inputs.TINY.N * inputs.TINY.steps + 1) * inputs.TINY.n,
                                                        dtype=torch.float64, device="cuda"))
        finally:
            dense.close()
    S.close()
