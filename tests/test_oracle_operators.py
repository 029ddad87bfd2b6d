"""Pins of the oracle's forcing-formulation operators (eq. 5, eq. 10) against
their definitions built densely in numpy, adjoint identities and the
spectrum of A."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import dense_A, oracle_problem

SMALL_AD = inputs.scaled(inputs.TINY, n=16, N=4, k=4, l=2, obs_stride=3)
SMALL_L96 = inputs.L96.replace(name="l96_small", n=20, N=3, steps=2, obs_stride=4, k=4, l=2)


def _l96_problem(cfg=SMALL_L96, seed=0):
    xb = cfg.F + np.random.default_rng(seed).standard_normal(cfg.n)
    return oracle_problem(cfg, xb=xb)


def _problems():
    return [oracle_problem(SMALL_AD, "stepping"), oracle_problem(SMALL_AD, "dense"), _l96_problem()]


def _circ(row):
    n = len(row)
    return row[(np.arange(n)[None, :] - np.arange(n)[:, None]) % n]


def _dense_parts(p):
    """Dense M_t (via the model on unit vectors), L, D^{1/2}, H, R^{-1} from their
    definitions (Section 2)."""
    n, N = p.n, p.N
    Ms = [np.stack([oracle.model_apply(p, t, e) for e in np.eye(n)], axis=1) for t in range(N)]
    L = np.eye(p.nA)
    for t in range(N):   # (L w)_{t+1} = w_{t+1} - M_t w_t
        L[(t + 1) * n:(t + 2) * n, t * n:(t + 1) * n] = -Ms[t]
    D = np.zeros((p.nA, p.nA))
    for t in range(N + 1):
        D[t * n:(t + 1) * n, t * n:(t + 1) * n] = _circ(p.Bsqrt if t == 0 else p.Qsqrt)
    rows = [t * n + s for t in range(N + 1) if t >= p.s.obs_t0 for s in range(0, n, p.s.obs_stride)]
    H = np.zeros((len(rows), p.nA))
    H[np.arange(len(rows)), rows] = 1.0
    return Ms, L, D, H


@pytest.mark.parametrize("pi", [0, 1, 2])
def test_model_adjoint(pi):
    p = _problems()[pi]
    g = np.random.default_rng(pi)
    for t in range(p.N):
        x, y = g.standard_normal(p.n), g.standard_normal(p.n)
        a = oracle.model_apply(p, t, x) @ y
        b = x @ oracle.model_apply(p, t, y, transpose=True)
        assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("pi", [0, 1, 2])
def test_Linv_adjoint_and_inverse(pi):
    """<L^{-1} x, y> = <x, L^{-T} y> and L (L^{-1} x) = x (eq. 5)."""
    p = _problems()[pi]
    g = np.random.default_rng(10 + pi)
    X, V = g.standard_normal((3, p.nA)), g.standard_normal((3, p.nA))
    W, S = oracle.Linv(p, X), oracle.LinvT(p, V)
    for j in range(3):
        a, b = W[j] @ V[j], X[j] @ S[j]
        assert abs(a - b) <= 1e-12 * abs(a)
    _, L, _, _ = _dense_parts(p)
    for j in range(3):
        assert np.linalg.norm(L @ W[j] - X[j]) <= 1e-13 * np.linalg.norm(X[j]) * 10


@pytest.mark.parametrize("pi", [0, 1, 2])
def test_A_matches_dense_definition(pi):
    """A = I + D^{1/2} L^{-T} H^T R^{-1} H L^{-1} D^{1/2} (eq. 10), with L^{-1}
    obtained by dense inversion of L (not by the recursion)."""
    p = _problems()[pi]
    _, L, D, H = _dense_parts(p)
    Li = np.linalg.inv(L)
    Aref = np.eye(p.nA) + D @ Li.T @ H.T @ H @ Li @ D / p.s.sigma_o2
    A = dense_A(p)
    assert np.abs(A - Aref).max() <= 1e-11 * np.abs(Aref).max()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()


def test_spectrum_of_A_tiny_config():
    """n_A - q eigenvalues equal to one and q larger ones (Section 2.2)."""
    cfg = inputs.TINY
    p = oracle_problem(cfg)
    A = dense_A(p)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert lam.min() == pytest.approx(1.0, abs=1e-10)
    q = p.nobs
    assert q == cfg.nobs == 100
    assert np.sum(np.abs(lam - 1.0) < 1e-8) == p.nA - q
    assert np.sum(lam > 1.0 + 1e-8) == q


def test_spectrum_of_A_paper_advection_size():
    """The paper's advection size (n=40, N=50, 2040 x 2040, 100 observations,
    Section 5.1) with the configured advection-diffusion physics."""
    cfg = inputs.scaled(inputs.TINY, n=40, N=50, k=25, l=5, obs_stride=4, steps=1, obs_t0=5)
    bs, _, _ = oracle.cov_sqrt_row(0, 40, 10.0, 0.1 ** 2)
    qs, _, _ = oracle.cov_sqrt_row(0, 40, 10.0, 0.05 ** 2)
    p = oracle.Problem(40, 50, oracle.MODEL_ADVDIFF, bs, qs, 0.05 ** 2, 4, obs_t0=5, obs_tstride=5,
                       steps=1, dt=0.02, kappa=1e-3, u=0.8)
    assert p.nA == 2040 and p.nobs == 100
    A = dense_A(p)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert lam.min() == pytest.approx(1.0, abs=1e-9)
    # A - I has rank <= q: at least n_A - q unit eigenvalues, and the q largest
    # carry the whole trace of A - I (some may be numerically close to one
    # because D^{1/2} has tiny eigenvalues at the shortest waves)
    assert np.sum(np.abs(lam - 1.0) < 1e-8) >= 2040 - 100
    assert np.sum(lam > 1.0 + 1e-8) <= 100
    assert np.sum(lam[-100:] - 1.0) == pytest.approx(np.trace(A) - 2040, rel=1e-10)


@pytest.mark.parametrize("pi", [1, 2])
def test_rhs_innovation_and_qcf(pi):
    """rhs = D^{1/2} L^{-T} H^T R^{-1} d (eq. 10, b = 0); d = y - H x;
    J (eq. 4) = 1/2 x^T A x - rhs^T x + J(0)."""
    p = _problems()[pi]
    Ms, L, D, H = _dense_parts(p)
    g = np.random.default_rng(20 + pi)
    xb = g.standard_normal(p.n) + (8.0 if p.model == oracle.MODEL_L96 else 0.0)
    y = g.standard_normal(p.nobs)
    d = oracle.innovation(p, xb, y)
    if p.model != oracle.MODEL_L96:   # linear model: x_t = M_{t-1}...M_0 xb
        xs = [xb]
        for t in range(p.N):
            xs.append(Ms[t] @ xs[-1])
        assert np.allclose(d, y - H @ np.concatenate(xs), atol=1e-12)
    r = oracle.rhs(p, d)
    Li = np.linalg.inv(L)
    assert np.allclose(r, D @ Li.T @ H.T @ d / p.s.sigma_o2, atol=1e-11 * np.abs(r).max())
    x = g.standard_normal(p.nA)
    A = dense_A(p)
    j0 = 0.5 * d @ d / p.s.sigma_o2
    jref = 0.5 * x @ x + 0.5 * np.sum((H @ Li @ D @ x - d) ** 2) / p.s.sigma_o2
    assert oracle.qcf(p, x, d) == pytest.approx(jref, rel=1e-12)
    assert oracle.qcf(p, x, d) == pytest.approx(0.5 * x @ A @ x - r @ x + j0, rel=1e-10)
