"""The paper's linear advection window (Section 5.1) built through the C-ABI
with a user-supplied upwind propagator: its Hessian products match the
oracle's on the same operator, and its spectrum has the structure the paper
states below eq. 10 -- every eigenvalue at least 1, and at most q of them
above 1 (A - I has rank <= q)."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import paper_setups as ps

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

_ctx = {}


def ctx():
    if "c" not in _ctx:
        _ctx["c"] = ps.advection_window(seed=0)
    return _ctx["c"]


def upwind_by_stepping(n, courant):
    """The oracle side's propagator: one upwind step applied to each unit
    vector, u_i <- u_i - C (u_i - u_{i-1}) with periodic u_{-1} = u_{n-1}."""
    M = np.zeros((n, n))
    for j in range(n):
        u = np.zeros(n)
        u[j] = 1.0
        M[:, j] = u - courant * (u - np.roll(u, 1))
    return M


def oracle_problem():
    n, N = ps.n_ADV, ps.N_ADV
    bs, _, _ = oracle.cov_sqrt_row(0, n, 10.0, 0.1 ** 2)      # SOAR, 10 dz
    qs, _, _ = oracle.cov_sqrt_row(0, n, 10.0, 0.05 ** 2)
    return oracle.Problem(n=n, N=N, model=oracle.MODEL_DENSE, Bsqrt=bs, Qsqrt=qs, sigma_o2=0.05 ** 2,
                          obs_stride=4, obs_t0=5, obs_tstride=5, steps=1, dt=1.0 / N,
                          M=upwind_by_stepping(n, 0.8), M_shared=True)


def test_upwind_window_hvp_matches_oracle():
    c = ctx()
    p = oracle_problem()
    nA = ps.n_ADV * (ps.N_ADV + 1)
    X = np.random.default_rng(3).standard_normal((6, nA))
    Y = torch.zeros(6, nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(c, torch.as_tensor(X, device="cuda"), Y, 6, nA, w.FP64)
    ref = oracle.hvp(p, X)
    assert np.abs(Y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert w.wc4d_nobs(c) == 100


def test_spectrum_matches_oracle_dense_A():
    """The whole spectrum of the library's A against the oracle's dense A on
    the same window.  A - I = D^{1/2} L^{-T} H^T R^{-1} H L^{-1} D^{1/2} has
    rank at most q = 100; here D^{1/2} is singular (the wrapped 40-point
    SOAR has 19 negative eigenvalues, clamped to zero), so fewer directions
    see the observations: the count of eigenvalues above one is the oracle's
    (60), every other eigenvalue is one, and the leading ones agree."""
    c = ctx()
    nA = ps.n_ADV * (ps.N_ADV + 1)
    A = ps.dense_A(c, nA)
    assert np.abs(A - A.T).max() <= 1e-10 * np.abs(A).max()
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    p = oracle_problem()
    Ao = oracle.hvp(p, np.eye(nA)).T
    lam_o = np.linalg.eigvalsh(0.5 * (Ao + Ao.T))
    above, above_o = np.sum(lam > 1.0 + 1e-8), np.sum(lam_o > 1.0 + 1e-8)
    assert above == above_o and 0 < above <= 100
    assert lam[0] >= 1.0 - 1e-10
    assert np.sum(np.abs(lam - 1.0) <= 1e-8) == nA - above
    assert np.abs(lam - lam_o).max() <= 1e-11 * lam_o.max()


def test_lambda_min_through_invariant_subspace_matches_dense():
    """The smallest eigenvalue of C^T A C from the rank argument (A - I has
    rank <= q, C - I rank <= k) equals the dense eigendecomposition's."""
    c = ctx()
    nA = ps.n_ADV * (ps.N_ADV + 1)
    k = 6
    w.wc4d_sketch(c, w.REVD, k, 4, 0, 9, None, w.FP64)
    U = torch.zeros(k, nA, dtype=torch.float64, device="cuda")
    th = w.wc4d_get_ritz(c, U, k)
    Uh = U.cpu().numpy()
    lam_sub = ps._lambda_min_CAC(c, nA, 100, Uh, th)
    A = ps.dense_A(c, nA)
    cc = 1.0 - 1.0 / np.sqrt(th)
    C = np.eye(nA) - (Uh.T * cc) @ Uh
    lam_dense = np.linalg.eigvalsh(C @ (0.5 * (A + A.T)) @ C).min()
    assert abs(lam_sub - lam_dense) <= 1e-9 * max(1.0, abs(lam_dense))


def test_lorenz96_paper_window_study_runs():
    r = ps.lorenz96_study(iters=3, seeds=(0,))
    assert r["nA"] == 80 * 151 and r["nobs"] == 120
    assert 0 < r["inner_loop_1"]["cg_iters"] <= 100
    for m in ("none", "deterministic", "revd", "nystrom", "ritzit"):
        assert len(r["qcf_decrease"][m]) == 3
        assert np.all(np.diff(r["qcf_decrease"][m]) > 0)     # CG decreases the quadratic cost
    for m, v in r["lambda_min_CAC"].items():
        assert v <= 1.0 + 1e-9


@pytest.mark.parametrize("obs,q", [(5, 480), (2, 3000)])
def test_lorenz96_denser_networks(obs, q):
    """Section 5.2's denser networks (every 5th variable at every 5th step:
    480 observations; every 2nd at every 2nd: 3000), k = 5 with the
    deterministic LMP of k = 15 pairs: observation counts, monotone
    quadratic-cost decrease, and (480 observations) lambda_min(C^T A C) <= 1
    for every LMP."""
    r = ps.lorenz96_study(k=5, l=5, iters=3, seeds=(0,), obs=obs, k_det=15, lmin=(q == 480))
    assert r["nobs"] == q and r["k_deterministic"] == 15
    for m in ("none", "deterministic", "revd", "nystrom", "ritzit"):
        assert np.all(np.diff(r["qcf_decrease"][m]) > 0)
    for m, v in r["lambda_min_CAC"].items():
        assert v <= 1.0 + 1e-9
