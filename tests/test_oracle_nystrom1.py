"""Pins of the oracle's single-pass Nystrom method (Tropp, Yurtsever, Udell,
Cevher 2017; the paper's Section 6 names single-pass Nystrom as future
work) against properties the mathematics fixes: exact recovery of a PSD
matrix whose rank does not exceed the sketch size, the Loewner bound
A_hat <= A (so every eigenvalue of the approximation is at most the matching
eigenvalue of A), and, for the 4D-Var operator of a tiny window, agreement
of the leading eigenvalue with a dense eigendecomposition of A."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem, dense_A


def _psd(n, lam, seed):
    g = np.random.default_rng(seed)
    V, _ = np.linalg.qr(g.standard_normal((n, len(lam))))
    return (V * lam) @ V.T


def test_exact_recovery_of_low_rank_psd():
    n, m, k = 60, 10, 6
    lam = np.array([50.0, 20.0, 9.0, 4.0, 2.0, 1.0])
    A = _psd(n, lam, 1)
    G = np.random.default_rng(2).standard_normal((m, n))
    U, th = oracle.nystrom_single_pass_core(lambda X: X @ A.T, G, k, 2.0 ** -52 * np.sqrt(n))
    assert np.allclose(th, lam, rtol=1e-10)
    Ahat = (U.T * th) @ U
    assert np.linalg.norm(Ahat - A) <= 1e-9 * np.linalg.norm(A)
    assert np.allclose(U @ U.T, np.eye(k), atol=1e-12)


def test_loewner_bound_on_full_rank_spd():
    n, m = 80, 12
    lam = 1.0 + 100.0 * 0.6 ** np.arange(n)
    A = _psd(n, lam, 3)
    G = np.random.default_rng(4).standard_normal((m, n))
    U, th = oracle.nystrom_single_pass_core(lambda X: X @ A.T, G, m, 2.0 ** -52 * np.sqrt(n))
    w = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.all(th <= w[:m] * (1 + 1e-12))
    # the approximation is dominated by A: A - A_hat is positive semi-definite
    Ahat = (U.T * th) @ U
    assert np.linalg.eigvalsh(A - Ahat).min() >= -1e-10 * w[0]


def test_4dvar_leading_eigenvalue_tiny_window():
    cfg = inputs.TINY
    p = oracle_problem(cfg, mode="stepping")
    A = dense_A(p)
    w = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))[::-1]
    G = inputs.probes(3, cfg.nA, cfg.k + cfg.l)
    U, th = oracle.nystrom_single_pass(p, cfg.k, G)
    assert np.all(th <= w[:cfg.k] * (1 + 1e-10))
    assert th[0] >= 0.9 * w[0]
    assert np.all(np.diff(th) <= 0)
