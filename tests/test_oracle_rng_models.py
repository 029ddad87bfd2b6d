"""Pins of the oracle's random numbers, covariance rows and models against
published values, closed forms and independent library routes."""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.integrate import solve_ivp

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Published known-answer vectors of Philox4x32-10 (Salmon et al. 2011)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_philox_words_are_counter_stream():
    w = oracle.philox_words(0x1234_5678_9ABC, 3)
    for c in range(3):
        ref = oracle.philox4x32_10([c, 0, 0, 0], [0x5678_9ABC, 0x1234])
        assert w[4 * c:4 * c + 4].tolist() == ref.tolist()


def test_gaussian_probes_are_standard_normal():
    """Alg. 3-5 step 1 wants i.i.d. N(0,1) entries."""
    G = oracle.gaussian(2024, 40_001, 5).ravel()
    assert abs(G.mean()) < 0.01
    assert abs(G.var() - 1.0) < 0.01
    ks = stats.kstest(G, "norm")
    assert ks.pvalue > 1e-3
    # the two Box-Muller outputs of one counter are uncorrelated
    pairs = G[: (len(G) // 2) * 2].reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.02


def test_gaussian_layout_and_seed():
    a = oracle.gaussian(7, 33, 3)
    b = oracle.gaussian(7, 33, 3)
    c = oracle.gaussian(8, 33, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # column-major element e = col*rows + row uses counter e >> 1
    flat = oracle.gaussian(7, 99, 1).ravel()
    assert np.array_equal(a.ravel(), flat)


# ---------------------------------------------------------------- covariances
def test_corr_rows_closed_forms():
    n, L = 64, 5.0
    s = oracle.corr_row(0, n, L, 2.0)
    assert s[0] == pytest.approx(2.0)
    assert s[5] == pytest.approx(2.0 * 2.0 / math.e, rel=1e-14)          # SOAR at r = L
    assert s[n - 5] == pytest.approx(s[5], rel=1e-15)                    # periodic distance
    g = oracle.corr_row(1, n, 4.0, 0.5)
    assert g[4] == pytest.approx(0.5 * math.exp(-0.5), rel=1e-14)        # Gaussian at r = L
    d = oracle.corr_row(2, n, 1.0, 0.05)
    assert d[0] == 0.05 and np.all(d[1:] == 0)


def _circ(row):
    n = len(row)
    idx = (np.arange(n)[None, :] - np.arange(n)[:, None]) % n
    return row[idx]


def _mp_eigs(kind, n, L, variance, dps=50):
    """Eigenvalues of the periodic-distance correlation circulant by a DFT of
    the correlation function evaluated at `dps` digits (mpmath): an
    independent, rounding-free statement of the definition."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp.clone() if hasattr(mpmath.mp, "clone") else mpmath.mp
    mp.dps = dps
    Lm = mp.mpf(L)
    row = []
    for s in range(n):
        r = mp.mpf(min(s, n - s))
        row.append((1 + r / Lm) * mp.exp(-r / Lm) if kind == 0 else mp.exp(-r * r / (2 * Lm * Lm)))
    cosv = [mp.cos(2 * mp.pi * j / n) for j in range(n)]
    return np.array([float(variance * mp.fsum(row[s] * cosv[(m * s) % n] for s in range(n))) for m in range(n)])


@pytest.mark.parametrize("kind,n,L", [(0, 64, 5.0), (0, 40, 10.0), (0, 63, 2.5), (1, 64, 4.0), (1, 63, 0.7),
                                      (1, 64, 20.0), (1, 128, 4.0), (1, 50, 1.5)])
def test_cov_eigs_match_high_precision_dft(kind, n, L):
    """Every eigenvalue, the smallest and the negative ones included, against
    a 50-digit DFT of the correlation function: relative 1e-14 for those
    above 1e-6 of the largest, and absolute 1e-17 of the largest below (SOAR
    is summed from its row in long double; the Gaussian's Poisson form has
    relative accuracy even at 1e-35)."""
    ref = _mp_eigs(kind, n, L, 0.7)
    lam = oracle.cov_eigs(kind, n, L, 0.7)
    big = np.abs(ref) > 1e-6 * ref.max()
    assert np.all(np.abs(lam - ref)[big] <= 1e-14 * np.abs(ref)[big])
    assert np.all(np.abs(lam - ref)[~big] <= 1e-17 * ref.max())
    if kind == 1:       # all-positive Poisson terms: relative accuracy everywhere it is positive
        pos = ref > 1e-300
        assert np.all(np.abs(lam - ref)[pos] <= 1e-12 * np.abs(ref)[pos] + 1e-20 * ref.max())
        assert np.array_equal(lam < 0, ref < 0)       # the clamping decisions agree


@pytest.mark.parametrize("kind,n,L", [(0, 100, 5.0), (0, 1024, 20.48), (0, 4096, 81.92), (1, 128, 4.0),
                                      (1, 8192, 4.0), (2, 50, 1.0)])
def test_cov_sqrt_squares_to_covariance(kind, n, L):
    """Positive-definite covariances (every eigenvalue > 0, nothing clamped):
    (C^{1/2})^2 = C to 1e-13 of the largest eigenvalue, in the Fourier basis
    (every circulant is diagonal there) and, for n <= 256, as dense matrices;
    the spectrum of the root is the square root of C's, mode by mode."""
    row = oracle.corr_row(kind, n, L, 0.7)
    srow, clamped, mn = oracle.cov_sqrt_row(kind, n, L, 0.7)
    lam = np.fft.fft(row).real
    assert clamped == 0 and mn > 0.0
    sig = np.fft.fft(srow).real                          # eigenvalues of the root
    assert np.abs(sig ** 2 - lam).max() <= 1e-13 * lam.max()
    assert np.all(sig > -1e-15 * np.sqrt(lam.max()))
    if n <= 256:
        C, S = _circ(row), _circ(srow)
        assert np.allclose(S, S.T, atol=1e-15)
        assert np.abs(S @ S - C).max() <= 1e-13 * lam.max()
    # every mode, the ones below 1e-8 of the largest included, against the
    # accurate eigenvalues (the square root is ill-conditioned only through
    # the rounding of the transform of the root's row, ~1e-16 of its largest)
    ex = np.sqrt(np.maximum(oracle.cov_eigs(kind, n, L, 0.7), 0.0))
    assert np.abs(sig - ex).max() <= 1e-14 * ex.max()


def test_cov_sqrt_clamps_only_negative_eigenvalues():
    """A periodically wrapped SOAR with a long length scale (40 points,
    L = 10, the paper's advection window) and a Gaussian whose truncated
    images make the highest wavenumbers slightly negative: the root squares
    to C with exactly the negative part of its spectrum removed, and the
    clamp count is the number of negative eigenvalues (taken from the
    50-digit DFT)."""
    for kind, n, L in [(0, 40, 10.0), (0, 256, 20.48), (1, 64, 4.0)]:
        ref = _mp_eigs(kind, n, L, 0.7)
        srow, clamped, mn = oracle.cov_sqrt_row(kind, n, L, 0.7)
        assert clamped == int(np.sum(ref < 0)) > 0
        assert mn == pytest.approx(ref.min(), rel=1e-9)
        C_pos = np.real(np.fft.ifft(np.maximum(ref, 0.0)))      # first row of C with the negative part removed
        S = _circ(srow)
        assert np.abs(S @ S - _circ(C_pos)).max() <= 1e-13 * ref.max()
    # the same from an explicit row (extended-precision DFT of the row)
    row = oracle.corr_row(0, 40, 10.0, 0.7)
    srow2, clamped2, _ = oracle.circulant_sqrt_row(row)
    srow1, clamped1, _ = oracle.cov_sqrt_row(0, 40, 10.0, 0.7)
    assert clamped2 == clamped1 and np.abs(srow2 - srow1).max() <= 1e-14 * np.abs(srow1).max()


def test_circulant_apply_matches_fft_convolution():
    g = np.random.default_rng(3)
    row = oracle.corr_row(0, 96, 7.0, 1.3)
    x = g.standard_normal(96)
    ref = np.real(np.fft.ifft(np.fft.fft(row) * np.fft.fft(x)))
    assert np.allclose(oracle.circulant_apply(row, x), ref, atol=1e-13)


# ---------------------------------------------------------------- advection-diffusion
def _cn_dense(n, kappa, u, dt):
    dz = 1.0 / n
    al, be, ga = kappa / dz**2 + u / (2 * dz), -2 * kappa / dz**2, kappa / dz**2 - u / (2 * dz)
    K = np.zeros((n, n))
    for s in range(n):
        K[s, (s - 1) % n] += al
        K[s, s] += be
        K[s, (s + 1) % n] += ga
    return K


@pytest.mark.parametrize("n", [8, 100, 257])
def test_cn_step_solves_the_crank_nicolson_system(n):
    kappa, u, dt = 1e-3, 0.5, 0.01
    K = _cn_dense(n, kappa, u, dt)
    x = np.random.default_rng(n).standard_normal(n)
    y = oracle.advdiff_step(x, kappa, u, dt)
    lhs = (np.eye(n) - 0.5 * dt * K) @ y
    rhs = (np.eye(n) + 0.5 * dt * K) @ x
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    v = np.random.default_rng(n + 1).standard_normal(n)
    yt = oracle.advdiff_step(v, kappa, u, dt, transpose=True)
    assert abs(y @ v - x @ yt) < 1e-13 * abs(y @ v) + 1e-13


@pytest.mark.parametrize("n,steps", [(100, 10), (64, 3), (4096, 10)])
def test_dense_propagator_matches_fourier_symbol(n, steps):
    """The CN step is circulant: its Fourier eigenvalue is
    (1 + dt/2 k_m) / (1 - dt/2 k_m), k_m = kappa (2cos th - 2)/dz^2 - i u sin th / dz."""
    kappa, u, dt = 1e-3, 0.5, 0.01
    if n == 4096:  # dense build at full size: check one column's spectrum only
        e0 = np.zeros(n); e0[0] = 1.0
        col = e0
        for _ in range(steps):
            col = oracle.advdiff_step(col, kappa, u, dt)
    else:
        M = oracle.advdiff_dense(n, kappa, u, dt, steps)
        col = M[:, 0]
        # circulant: every column is the shifted first column
        for c in (1, n // 2, n - 1):
            assert np.allclose(M[:, c], np.roll(col, c), atol=1e-14)
    dz = 1.0 / n
    th = 2 * np.pi * np.arange(n) / n
    khat = kappa * (2 * np.cos(th) - 2) / dz**2 - 1j * u * np.sin(th) / dz
    g = ((1 + 0.5 * dt * khat) / (1 - 0.5 * dt * khat)) ** steps
    lam = np.fft.fft(col)
    assert np.abs(lam - g).max() < 1e-12


# ---------------------------------------------------------------- Lorenz-96
def test_l96_fixed_point():
    x = np.full(40, 8.0)
    assert np.abs(oracle.l96_tendency(x, 8.0)).max() == 0.0
    assert np.array_equal(oracle.l96_rk4(x, 8.0, 0.025), x)


def test_l96_rk4_is_fourth_order():
    n, F, T = 40, 8.0, 0.4
    x0 = F + 0.5 * np.random.default_rng(1).standard_normal(n)
    f = lambda _t, x: (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F
    ref = solve_ivp(f, (0, T), x0, method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for nsteps in (8, 16, 32):
        traj = oracle.l96_run(x0, F, T / nsteps, nsteps)
        errs.append(np.abs(traj[-1] - ref).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, errs


def test_l96_tlm_taylor_and_adjoint():
    n, F, dt = 36, 8.0, 0.025
    g = np.random.default_rng(5)
    x = F + g.standard_normal(n)
    d = g.standard_normal(n)
    base = oracle.l96_rk4(x, F, dt)
    tl = oracle.l96_tlm(x, d, F, dt)
    prev = None
    for eps in (1e-1, 1e-2, 1e-3, 1e-4):
        r = np.linalg.norm(oracle.l96_rk4(x + eps * d, F, dt) - base - eps * tl)
        if prev is not None:
            assert 50 < prev / r < 200   # O(eps^2) remainder
        prev = r
    ly = g.standard_normal(n)
    lx = oracle.l96_adj(x, ly, F, dt)
    assert abs(tl @ ly - d @ lx) < 1e-13 * abs(tl @ ly)


# ---------------------------------------------------------------- paper sizes
def test_paper_problem_sizes_and_observation_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for c in g["cases"]:
        row = np.zeros(c["n"]); row[0] = 1.0
        p = oracle.Problem(c["n"], c["N"], oracle.MODEL_ADVDIFF, row, row, 1.0, c["obs_stride"],
                           obs_t0=c["obs_t0"], obs_tstride=c["obs_tstride"])
        assert p.nA == c["nA"], c["cite"]
        assert p.nobs == c["q"], c["cite"]
