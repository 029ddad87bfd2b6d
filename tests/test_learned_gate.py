"""The learned-proposal gate (host logic, no GPU): top-k Ritz sums compared
at ratio 1 by default, Ky Fan's bound as the reason, non-finite values
rejected."""
import numpy as np
import pytest

from paper_2101_07249_gb300.learned import accept


def test_gate_compares_top_k_ritz_sums():
    g = np.array([100.0, 50.0, 10.0, 2.0])
    assert accept(g, g)                                   # equal blocks: accepted at ratio 1
    assert not accept(g * 0.999, g)                       # any loss: Gaussian fallback
    assert accept([120.0, 45.0, 1.0, 1.0], g, k=2)        # 165 >= 150
    assert accept([120.0, 40.0, 1.0, 1.0], g)             # 162 >= 162
    assert not accept([120.0, 39.0, 1.0, 1.0], g)         # 161 < 162
    assert accept([101.0, 50.0, 10.0, 2.0], g, ratio=1.0)
    assert accept(g * 0.95, g, ratio=0.9)


def test_gate_rejects_non_finite_and_short_input():
    g = np.array([3.0, 2.0, 1.0])
    assert not accept([np.nan, 2.0, 1.0], g)
    assert not accept([np.inf, 2.0, 1.0], [np.inf, 2.0, 1.0])
    with pytest.raises(ValueError):
        accept([1.0], g, k=2)


def test_ky_fan_bound_makes_the_sum_a_subspace_score():
    """On a random SPD matrix, the top-k Ritz sum of a subspace containing
    the leading invariant subspace equals the top-k eigenvalue sum and beats
    a random subspace of the same width."""
    rng = np.random.default_rng(0)
    n, k, m = 60, 5, 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(1, 100, n))[::-1]
    A = (Q * lam) @ Q.T

    def ritz(V):
        V, _ = np.linalg.qr(V)
        return np.sort(np.linalg.eigvalsh(V.T @ A @ V))[::-1]

    good = np.hstack([Q[:, :k], rng.standard_normal((n, m - k))])
    rand = rng.standard_normal((n, m))
    assert np.sum(ritz(good)[:k]) == pytest.approx(np.sum(lam[:k]), rel=1e-12)
    assert accept(ritz(good), ritz(rand), k=k)
    assert not accept(ritz(rand), ritz(good), k=k)
