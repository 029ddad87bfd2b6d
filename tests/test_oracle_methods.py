"""Pins of the oracle's dense linear algebra, the three randomised
eigensolvers (Alg. 3-5), the spectral LMP (eq. 14-16) and PCG (Alg. 1)
against numpy/scipy, subspace definitions and the properties the paper
states."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import dense_A, oracle_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------- dense LA
def test_householder_qr():
    g = np.random.default_rng(0)
    A = g.standard_normal((7, 50))           # 7 columns of length 50
    Q, R = oracle.householder_qr(A)
    assert np.allclose(Q @ Q.T, np.eye(7), atol=1e-14)
    assert np.allclose(R.T @ Q, A, atol=1e-13)    # columns: A_j = sum_i Q_i R_ij
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    Qn, Rn = np.linalg.qr(A.T)
    sgn = np.sign(np.diag(Rn))
    assert np.allclose(Q.T, Qn * sgn, atol=1e-13)


@pytest.mark.parametrize("m", [1, 5, 40])
def test_jacobi_eig(m):
    g = np.random.default_rng(m)
    X = g.standard_normal((m, m))
    A = X @ X.T + np.diag(np.arange(m))
    w, V, sweeps = oracle.jacobi_eig(A)
    assert sweeps >= 0
    wn = np.linalg.eigvalsh(A)[::-1]
    assert np.allclose(w, wn, rtol=1e-13, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(m), atol=1e-13)
    assert np.allclose(A @ V, V * w, atol=1e-11 * np.abs(A).max())


def test_cholesky_and_triangular_solve():
    g = np.random.default_rng(3)
    X = g.standard_normal((30, 9))
    A = X.T @ X
    R, rc = oracle.cholesky_upper(A)
    assert rc == 0
    assert np.allclose(R, np.linalg.cholesky(A).T, atol=1e-12)
    B = g.standard_normal((40, 9))
    F = oracle.solve_right_upper(B, R)
    assert np.allclose(F @ R, B, atol=1e-12)
    A2 = A.copy(); A2[4, 4] = -1.0
    assert oracle.cholesky_upper(A2)[1] > 0


def test_jacobi_svd():
    g = np.random.default_rng(4)
    A = g.standard_normal((60, 8)) @ np.diag(np.logspace(0, 3, 8))
    U, s, V, rc = oracle.jacobi_svd(A)
    assert rc >= 0
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
    assert np.allclose((U * s) @ V.T, A, atol=1e-11 * s[0])
    assert np.allclose(U.T @ U, np.eye(8), atol=1e-13)


# ------------------------------------------------------------- methods
CFG = inputs.TINY


@pytest.fixture(scope="module")
def tiny():
    p = oracle_problem(CFG)
    A = dense_A(p)
    A = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(A)
    return p, A, lam[::-1], V[:, ::-1]


def _orth(Y):
    Q, R = np.linalg.qr(Y)
    return Q * np.sign(np.diag(R))


def _lmp_dense(U, th):
    c = 1.0 - 1.0 / np.sqrt(th)
    return np.eye(U.shape[0]) - (U * c) @ U.T


def _check_same_pairs(U, th, Uref, thref, tol=1e-9):
    assert np.allclose(th, thref, rtol=tol)
    # sign/rotation-invariant comparison: the LMP factor built from the pairs
    C, Cref = _lmp_dense(U.T, th), _lmp_dense(Uref, thref)
    assert np.abs(C - Cref).max() < 1e3 * tol


def test_revd_is_rayleigh_ritz_on_power_subspace(tiny):
    """REVD(q) = Rayleigh-Ritz of A on span(A^{q+1} G) (Alg. 2-3)."""
    p, A, lam, _ = tiny
    k, m = CFG.k, CFG.K
    G = inputs.probes(1, p.nA, m)
    for q in (0, 1, 2):
        U, th = oracle.revd(p, k, G, q=q)
        Z = _orth(np.linalg.matrix_power(A, q + 1) @ G.T)
        w, W = np.linalg.eigh(Z.T @ A @ Z)
        _check_same_pairs(U, th, (Z @ W[:, ::-1])[:, :k], w[::-1][:k])
        assert np.all(th >= 1.0 - 1e-12) and np.all(th <= lam[:k] * (1 + 1e-12))   # interlacing


def test_nystrom_is_top_eigenpairs_of_nystrom_approximation(tiny):
    """Nystrom: top-k eigenpairs of A Z (Z^T A Z)^{-1} Z^T A, Z = orth(A G) (Alg. 4)."""
    p, A, lam, _ = tiny
    k, m = CFG.k, CFG.K
    G = inputs.probes(2, p.nA, m)
    U, th = oracle.nystrom(p, k, G)
    Z = _orth(A @ G.T)
    AZ = A @ Z
    An = AZ @ np.linalg.solve(Z.T @ AZ, AZ.T)
    w, W = np.linalg.eigh(0.5 * (An + An.T))
    _check_same_pairs(U, th, W[:, ::-1][:, :k], w[::-1][:k])
    assert np.all(th >= 1.0 - 1e-12) and np.all(th <= lam[:k] * (1 + 1e-10))


def test_ritzit_is_top_singular_triplets(tiny):
    """REVD_ritzit: Theta_3, U_3 = top-k singular values / left vectors of
    A G_3, G_3 = orth(G) (Alg. 5)."""
    p, A, lam, _ = tiny
    k, m = CFG.k, CFG.K
    G = inputs.probes(3, p.nA, m)
    U, th = oracle.ritzit(p, k, G)
    Us, s, _ = np.linalg.svd(A @ _orth(G.T), full_matrices=False)
    _check_same_pairs(U, th, Us[:, :k], s[:k])
    assert np.all(th >= 1.0 - 1e-12) and np.all(th <= lam[:k] * (1 + 1e-10))


def test_full_sketch_recovers_exact_eigenpairs():
    """With k + l = n_A every method returns exact eigenpairs."""
    cfg = inputs.scaled(inputs.TINY, n=10, N=3, k=6, l=34, obs_stride=2)
    p = oracle_problem(cfg)
    A = dense_A(p)
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    lam, V = lam[::-1], V[:, ::-1]
    G = inputs.probes(4, p.nA, p.nA)
    for name, (U, th) in {"revd": oracle.revd(p, 6, G, q=0), "nystrom": oracle.nystrom(p, 6, G),
                          "ritzit": oracle.ritzit(p, 6, G)}.items():
        assert np.allclose(th, lam[:6], rtol=1e-10), name
        # eigenpair residual (the tiny periodic grid has repeated eigenvalues,
        # so individual eigenvectors are not unique)
        assert np.abs(A @ U.T - U.T * th).max() <= 1e-9 * lam[0], name
        assert np.allclose(U @ U.T, np.eye(6), atol=1e-12), name


def test_products_with_A_match_table_1(tiny):
    p, _, _, _ = tiny
    tab = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["table1_products_with_A"]
    G = inputs.probes(5, p.nA, CFG.K)
    oracle.hvp_count(reset=True)
    oracle.revd(p, CFG.k, G, q=0)
    assert oracle.hvp_count(reset=True) == tab["revd"]
    oracle.revd(p, CFG.k, G, q=1)
    assert oracle.hvp_count(reset=True) == tab["revd"] + 1
    oracle.nystrom(p, CFG.k, G)
    assert oracle.hvp_count(reset=True) == tab["nystrom"]
    oracle.ritzit(p, CFG.k, G)
    assert oracle.hvp_count(reset=True) == tab["ritzit"]


# ------------------------------------------------------------- LMP
def test_lmp_factor_and_exact_eigenpairs(tiny):
    """Eq. 12-14 with exact eigenvectors: C C^T = P_sp = P_k; C^T A C has k
    unit eigenvalues and otherwise A's spectrum."""
    p, A, lam, V = tiny
    k = 12
    U, th = V[:, :k], lam[:k]
    Ut = np.ascontiguousarray(U.T)
    E = np.eye(p.nA)
    Cd = np.stack([oracle.lmp_apply(Ut, th, e) for e in E], axis=1)
    CTd = np.stack([oracle.lmp_apply(Ut, th, e, transpose=True) for e in E], axis=1)
    assert np.allclose(CTd, Cd.T, atol=1e-14)
    Psp = E - (U * (1.0 - 1.0 / th)) @ U.T                     # eq. 15
    assert np.allclose(Cd @ Cd.T, Psp, atol=1e-12)
    S = U                                                      # eq. 14 with S = V
    SAS = S.T @ A @ S
    Pk = (E - S @ np.linalg.solve(SAS, S.T @ A)) @ (E - A @ S @ np.linalg.solve(SAS, S.T)) \
        + S @ np.linalg.solve(SAS, S.T)
    assert np.allclose(Pk, Psp, atol=1e-9)
    mu = np.sort(np.linalg.eigvalsh(Cd.T @ A @ Cd))[::-1]
    assert np.sum(np.abs(mu - 1.0) < 1e-8) >= k + (p.nA - p.nobs)
    assert np.allclose(mu[: p.nobs - k], lam[k:p.nobs], rtol=1e-9)


def test_lmp_with_all_eigenpairs_is_inverse():
    cfg = inputs.scaled(inputs.TINY, n=8, N=2, k=2, l=2, obs_stride=2)
    p = oracle_problem(cfg)
    A = dense_A(p)
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    Ut = np.ascontiguousarray(V.T)
    Cd = np.stack([oracle.lmp_apply(Ut, lam, e) for e in np.eye(p.nA)], axis=1)
    assert np.allclose(Cd @ Cd.T, np.linalg.inv(A), atol=1e-12)


# ------------------------------------------------------------- PCG
def _rhs(p, cfg):
    tw = inputs.twin(cfg)
    d = oracle.innovation(p, tw.xb, tw.y)
    return d, oracle.rhs(p, d)


def test_pcg_matches_dense_solve_and_qcf(tiny):
    p, A, lam, V = tiny
    d, b = _rhs(p, CFG)
    xs = np.linalg.solve(A, b)
    for k in (0, 10):
        U = np.ascontiguousarray(V[:, :k].T) if k else None
        th = lam[:k] if k else None
        r = oracle.pcg(p, b, U, th, tol=1e-13, maxit=500)
        assert r["status"] == 0
        assert np.linalg.norm(r["x"] - xs) <= 1e-10 * np.linalg.norm(xs)
        # eq. 4 decreases at every iteration by alpha rho / 2
        assert np.all(r["qcf_drop"] > 0)
        j0 = oracle.qcf(p, np.zeros(p.nA), d)
        assert j0 - r["qcf_drop"].sum() == pytest.approx(oracle.qcf(p, r["x"], d), rel=1e-9)
    # finite termination: A has at most q + 1 distinct eigenvalues
    r = oracle.pcg(p, b, tol=1e-10, maxit=1000)
    assert r["iters"] <= p.nobs + 1
    U = np.ascontiguousarray(V[:, :10].T)
    r2 = oracle.pcg(p, b, U, lam[:10], tol=1e-10, maxit=1000)
    assert r2["iters"] <= p.nobs - 10 + 1


def test_pcg_error_bound_eq10(tiny):
    """|e_i|_A / |e_0|_A <= 2 ((sqrt k - 1)/(sqrt k + 1))^i (eq. 12)."""
    p, A, lam, _ = tiny
    _, b = _rhs(p, CFG)
    xs = np.linalg.solve(A, b)
    kappa = lam[0] / lam[-1]
    rate = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    e0 = np.sqrt(xs @ A @ xs)
    for i in (1, 3, 8, 20):
        x = oracle.pcg(p, b, force_iters=i)["x"]
        e = xs - x
        assert np.sqrt(e @ A @ e) / e0 <= 2 * rate ** i * (1 + 1e-9)


def test_pcg_reaches_tolerance_with_randomised_lmps(tiny):
    """The inner-loop procedure of Section 4: Ritz pairs from each method,
    spectral LMP, PCG on the exact A to relative residual 1e-6."""
    p, A, _, _ = tiny
    _, b = _rhs(p, CFG)
    G = inputs.probes(6, p.nA, CFG.K)
    base = oracle.pcg(p, b, tol=1e-6)
    for U, th in (oracle.revd(p, CFG.k, G, q=1), oracle.nystrom(p, CFG.k, G), oracle.ritzit(p, CFG.k, G)):
        r = oracle.pcg(p, b, U, th, tol=1e-6)
        assert r["status"] == 0 and r["relres"] <= 1e-6
        assert np.linalg.norm(b - A @ r["x"]) / np.linalg.norm(b) <= 2e-6
        assert r["iters"] <= base["iters"]
