"""Pins of the oracle's Lanczos Ritz pairs from CG (Section 3.3, eq. 18-20)
against what the mathematics fixes: with complete reorthogonalisation the
normalised residuals are orthonormal and F_J^T A F_J = T_J (the Lanczos
relation CG's coefficients encode), the Ritz values lie inside A's spectrum
and the largest converges to lambda_max(A) (dense eigendecomposition of the
tiny window's A), and a planted slip in gamma_j breaks the relation."""
import numpy as np

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem, dense_A

CFG = inputs.TINY


def _setup():
    p = oracle_problem(CFG, mode="stepping")
    tw = inputs.twin(CFG)
    b = oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))
    return p, b


def test_lanczos_relation_and_orthonormality():
    p, b = _setup()
    J = 20
    out = oracle.lanczos_cg(p, b, J, reorth=True)
    F = out["F"][:J]
    assert np.abs(F @ F.T - np.eye(J)).max() < 1e-12
    A = dense_A(p)
    T = oracle.lanczos_tridiag(out["alpha"], out["beta"])
    FAF = F @ A @ F.T
    assert np.abs(FAF - T).max() < 1e-9 * np.abs(T).max()


def test_ritz_values_inside_spectrum_and_top_converges():
    p, b = _setup()
    A = dense_A(p)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    out = oracle.lanczos_cg(p, b, 60, reorth=True)
    U, th = oracle.lanczos_ritz(out["alpha"], out["beta"], out["F"], 5)
    assert np.all(th <= lam[-1] * (1 + 1e-10)) and np.all(th >= lam[0] * (1 - 1e-10))
    assert abs(th[0] - lam[-1]) <= 1e-8 * lam[-1]
    # Ritz vectors: orthonormal, and A u = theta u approximately for the top pair
    assert np.abs(U @ U.T - np.eye(5)).max() < 1e-10
    r = A @ U[0] - th[0] * U[0]
    assert np.linalg.norm(r) < 1e-6 * th[0]


def test_planted_gamma_slip_breaks_the_relation():
    """gamma_j = 1/alpha_j alone (dropping beta_{j-1}/alpha_{j-1}) is a
    plausible slip; the Lanczos relation exposes it."""
    p, b = _setup()
    J = 12
    out = oracle.lanczos_cg(p, b, J, reorth=True)
    F = out["F"][:J]
    A = dense_A(p)
    T = oracle.lanczos_tridiag(out["alpha"], out["beta"])
    T_bad = T.copy()
    T_bad[np.arange(J), np.arange(J)] = 1.0 / out["alpha"]
    FAF = F @ A @ F.T
    assert np.abs(FAF - T).max() < 1e-9 * np.abs(T).max()
    assert np.abs(FAF - T_bad).max() > 1e-3 * np.abs(T).max()


def test_cg_iterates_match_oracle_pcg():
    """The recording CG is Alg. 1 with C = I: its iterate equals the oracle's
    own PCG without an LMP after the same few iterations (no
    reorthogonalisation; FP64 CG on this window drifts apart by rounding
    after ~10 iterations)."""
    p, b = _setup()
    out = oracle.lanczos_cg(p, b, 5, reorth=False)
    ro = oracle.pcg(p, b, None, None, force_iters=5)
    assert np.linalg.norm(out["x"] - ro["x"]) <= 1e-10 * np.linalg.norm(ro["x"])
