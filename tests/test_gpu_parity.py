"""Parity of the CUDA library (through the C-ABI) against the FP64 oracle on
the same seeded inputs, at sizes the oracle finishes in seconds: several
tiles and ragged tails, the direct (n = 100) and FFT (n = 128, 64) circulant
paths, the dense advection-diffusion and the Lorenz-96 models.

Tolerances: FP64 path 1e-10 relative on solutions and Ritz values (1e-12 on
single operator products); mixed path relative residual <= 1e-6 and solution
within 1e-5 of the oracle."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

AD_DIRECT = inputs.TINY                                                     # n = 100: direct circulant
AD_FFT = inputs.scaled(inputs.TINY, n=128, N=6, k=12, l=4, obs_stride=6)    # n = 128: FFT path
L96S = inputs.L96.replace(name="l96_n64_N4", n=64, N=4, steps=3, obs_stride=4, k=8, l=4)
CASES = {"ad_direct": AD_DIRECT, "ad_fft": AD_FFT, "l96": L96S}


def dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.double().cpu().numpy()


_cache = {}


def setup(name):
    if name not in _cache:
        cfg = CASES[name]
        tw = inputs.twin(cfg)
        S = w.Solver(cfg, tw)
        p = oracle_problem(cfg, mode="stepping", xb=tw.xb)
        _cache[name] = (cfg, S, p, tw)
    return _cache[name]


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


# ------------------------------------------------------------------ set-up pieces
def test_gaussian_matches_oracle():
    cfg, S, _, _ = setup("ad_direct")
    rows, cols = 1001, 3
    G = torch.zeros(cols, rows, dtype=torch.float64, device="cuda")
    w.wc4d_gaussian(S.ctx, 12345, rows, cols, rows, G)
    ref = oracle.gaussian(12345, rows, cols)
    assert np.abs(host(G) - ref).max() < 1e-13 * np.abs(ref).max()


def test_gaussian_f32_matches_oracle_to_fp32_rounding():
    """The mixed sketch's FP32 probes: the oracle's Philox stream and
    Box-Muller in FP64, against the same counters in FP32 arithmetic.  The
    uniforms are the FP32 roundings of the FP64 ones, so an entry differs by
    a few FP32 ulp of the log, sqrt, sin and cos -- except where u1 is within
    a few ulp of 1, where the radius sqrt(-2 log u1) is tiny in both and the
    difference stays below its own size."""
    cfg, S, _, _ = setup("ad_direct")
    rows, cols = 100003, 5                          # ragged: an odd total uses half a counter
    G = torch.zeros(cols, rows, dtype=torch.float32, device="cuda")
    w.wc4d_gaussian_f32(S.ctx, 777, rows, cols, rows, G)
    ref = oracle.gaussian(777, rows, cols)
    got = host(G).astype(np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= 1e-5 * np.maximum(np.abs(ref), 1.0) + 1e-3 * (np.abs(ref) < 1e-2))
    assert np.median(err / np.maximum(np.abs(ref), 1e-30)) < 3e-7
    assert abs(got.mean()) < 0.01 and abs(got.std() - 1.0) < 0.01


def test_propagator_matches_stepping():
    cfg, S, _, _ = setup("ad_fft")
    M = torch.zeros(cfg.n, cfg.n, dtype=torch.float64, device="cuda")
    w.wc4d_get_propagator(S.ctx, 0, M)
    ref = oracle.advdiff_dense(cfg.n, cfg.kappa, cfg.u, cfg.dt, cfg.steps)
    assert np.abs(host(M) - ref).max() < 1e-13
    w.wc4d_get_propagator(S.ctx, cfg.N - 1, M)
    assert np.abs(host(M) - ref).max() < 1e-13


@pytest.mark.parametrize("name", list(CASES))
def test_dsqrt_matches_oracle(name):
    cfg, S, p, _ = setup(name)
    X = inputs.block(1, cfg.nA, 5)
    Y = torch.zeros(5, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, dev(X), Y, 5, cfg.nA)
    assert colrel(host(Y), oracle.Dsqrt(p, X)) < 1e-12
    Y32 = torch.zeros(5, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, dev(X, torch.float32), Y32, 5, cfg.nA, w.MIXED)
    assert colrel(host(Y32), oracle.Dsqrt(p, X)) < 1e-5


@pytest.mark.parametrize("name", list(CASES))
def test_linv_and_linvT_match_oracle(name):
    cfg, S, p, _ = setup(name)
    X = inputs.block(2, cfg.nA, 3)
    W = dev(X)
    w.wc4d_apply_linv(S.ctx, W, 3, cfg.nA)
    assert colrel(host(W), oracle.Linv(p, X)) < 1e-12
    W = dev(X)
    w.wc4d_apply_linvT(S.ctx, W, 3, cfg.nA)
    assert colrel(host(W), oracle.LinvT(p, X)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("K", [1, 7, 20, 65])
def test_hvp_fp64_matches_oracle(name, K):
    cfg, S, p, _ = setup(name)
    X = inputs.block(3 + K, cfg.nA, K)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X), Y, K, cfg.nA, w.FP64)
    assert colrel(host(Y), oracle.hvp(p, X)) < 1e-12


def test_hvp_ragged_257_columns():
    cfg, S, p, _ = setup("ad_fft")
    K = 257
    X = inputs.block(9, cfg.nA, K)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X), Y, K, cfg.nA, w.FP64)
    ref = oracle.hvp(p, X)
    assert colrel(host(Y), ref) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("K", [1, 20])
def test_hvp_mixed_matches_oracle(name, K):
    cfg, S, p, _ = setup(name)
    X = inputs.block(30 + K, cfg.nA, K)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X, torch.float32), Y, K, cfg.nA, w.MIXED)
    assert colrel(host(Y), oracle.hvp(p, X)) < 2e-5


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(name):
    cfg, S, p, tw = setup(name)
    r = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_get_rhs(S.ctx, r)
    d = oracle.innovation(p, tw.xb, tw.y)
    assert relerr(host(r), oracle.rhs(p, d)) < 1e-12
    assert w.wc4d_nobs(S.ctx) == cfg.nobs == p.nobs


# ------------------------------------------------------------------ small dense LA
@pytest.mark.parametrize("m", [1, 6, 15, 33])
def test_cholqr2_matches_householder(m):
    cfg, S, _, _ = setup("ad_direct")
    g = np.random.default_rng(m)
    A = g.standard_normal((m, 600)) * np.logspace(0, 2, m)[:, None]
    Y = dev(A)
    R = w.wc4d_orthonormalize(S.ctx, Y, 600, m, 600)
    Qo, Ro = oracle.householder_qr(A)
    assert np.abs(host(Y) @ host(Y).T - np.eye(m)).max() < 1e-13
    assert relerr(R, Ro) < 1e-11
    assert np.abs(host(Y) - Qo).max() < 1e-9


@pytest.mark.parametrize("m", [64, 128, 200])
def test_cholqr2_fp32_ill_conditioned(m):
    """FP32 blocks (the mixed sketch's orthonormalisation) with condition
    number 1e5: the Gram matrix must carry ~FP64 accuracy (kappa^2 = 1e10
    exceeds what FP32 accumulation resolves), so CholeskyQR2 still returns
    orthonormal columns to FP32 rounding and Y = Z R."""
    cfg, S, _, _ = setup("ad_direct")
    rows = 20000
    g = np.random.default_rng(100 + m)
    Q1, _ = np.linalg.qr(g.standard_normal((rows, m)))
    V, _ = np.linalg.qr(g.standard_normal((m, m)))
    A = (Q1 * np.logspace(0, -5, m)) @ V.T            # rows x m, kappa = 1e5
    A32 = A.astype(np.float32).astype(np.float64)
    Y = torch.tensor(A32.T.copy(), dtype=torch.float32, device="cuda")
    R = w.wc4d_orthonormalize(S.ctx, Y, rows, m, rows, precision=w.MIXED)
    Z = host(Y).astype(np.float64).T
    assert np.abs(Z.T @ Z - np.eye(m)).max() < 2e-5
    assert np.linalg.norm(A32 - Z @ R) / np.linalg.norm(A32) < 1e-5
    assert np.all(np.diag(R) > 0)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_shifted_cholqr3_numerically_rank_deficient(precision):
    """A block whose singular values span 1e10 (FP32 data) or 1e15 (FP64):
    the Gram matrix is numerically singular (condition beyond 1e16), the
    unshifted Cholesky breaks down, and the shifted pass plus two more
    (shifted CholeskyQR3) still return orthonormal columns with Y = Z R."""
    cfg, S, _, _ = setup("ad_direct")
    rows, m = 8000, 48
    g = np.random.default_rng(7)
    Q1, _ = np.linalg.qr(g.standard_normal((rows, m)))
    V, _ = np.linalg.qr(g.standard_normal((m, m)))
    span = -10 if precision == "mixed" else -15
    A = (Q1 * np.logspace(0, span, m)) @ V.T
    dt = torch.float32 if precision == "mixed" else torch.float64
    A_in = A.astype(np.float32).astype(np.float64) if precision == "mixed" else A
    Y = torch.tensor(A_in.T.copy(), dtype=dt, device="cuda")
    R = w.wc4d_orthonormalize(S.ctx, Y, rows, m, rows, precision=w.MIXED if precision == "mixed" else w.FP64)
    Z = host(Y).T
    ortho, recon = (1e-4, 1e-5) if precision == "mixed" else (1e-11, 1e-12)
    assert np.abs(Z.T @ Z - np.eye(m)).max() < ortho
    assert np.linalg.norm(A_in - Z @ R) / np.linalg.norm(A_in) < recon


@pytest.mark.parametrize("m", [1, 2, 15, 40, 77])
def test_symeig_matches_jacobi(m):
    cfg, S, _, _ = setup("ad_direct")
    g = np.random.default_rng(100 + m)
    X = g.standard_normal((m, m))
    A = X @ X.T + np.eye(m)
    V = torch.zeros(m, m, dtype=torch.float64, device="cuda")
    wv = w.wc4d_symeig(S.ctx, m, dev(A.T), V)       # column-major = transpose of row-major
    wo, Vo, _ = oracle.jacobi_eig(A)
    assert np.allclose(wv, wo, rtol=1e-12, atol=1e-12)
    Vg = host(V).T                                   # columns = eigenvectors
    assert np.abs(A @ Vg - Vg * wv).max() < 1e-11 * wo[0]
    assert m < 2 or w.wc4d_jacobi_sweeps(S.ctx) >= 1


@pytest.mark.parametrize("method", ["revd", "nystrom", "ritzit", "nystrom1"])
def test_mixed_sketch_eigensolve_stops_early(method):
    """The small eigensolve of a mixed sketch stops after the sweep that
    brings the columns within |cos| <= 1e-5; the FP64 sketch runs to a sweep
    without rotations.  Both orderings converge quadratically, so the mixed
    one uses no more sweeps, and its Ritz values still agree to ~1e-5."""
    cfg, S, _, _ = setup("ad_fft")
    m = cfg.k + cfg.l
    w.wc4d_sketch(S.ctx, w.METHODS[method], cfg.k, cfg.l, cfg.q_power, 23, None, w.FP64)
    s64 = w.wc4d_jacobi_sweeps(S.ctx)
    U = torch.zeros(cfg.k, cfg.nA, dtype=torch.float64, device="cuda")
    th64 = w.wc4d_get_ritz(S.ctx, U, cfg.k)
    w.wc4d_sketch(S.ctx, w.METHODS[method], cfg.k, cfg.l, cfg.q_power, 23, None, w.MIXED)
    s32 = w.wc4d_jacobi_sweeps(S.ctx)
    th32 = w.wc4d_get_ritz(S.ctx, U, cfg.k)
    assert 1 <= s32 <= s64 <= 60
    # the FP32 pre-rotation (eigensolves of SPD matrices from their Cholesky
    # factor: not ritzit's SVD of R_3) ran on one 16-CTA cluster (a GB300
    # schedules clusters of 16 with 64 KB of shared memory each)
    if method != "ritzit":
        assert w.wc4d_jacobi_sweeps_fp32(S.ctx) != 0
        assert w.wc4d_jacobi_fp32_kernel(S.ctx) == 1
    assert np.allclose(th32, th64, rtol=1e-3)
    Ug = host(U)
    assert np.abs(Ug @ Ug.T - np.eye(cfg.k)).max() < 1e-4


# ------------------------------------------------------------------ eigensolvers
def oracle_pairs(method, p, k, G, q):
    """The oracle's Ritz pairs for a sketch method on the same probes."""
    if method == "revd":
        return oracle.revd(p, k, G, q=q)
    if method == "nystrom":
        return oracle.nystrom(p, k, G)
    if method == "nystrom1":
        return oracle.nystrom_single_pass(p, k, G)
    return oracle.ritzit(p, k, G)


def _lmp_dense(U, th):
    c = 1.0 - 1.0 / np.sqrt(th)
    return np.eye(U.shape[1]) - (U.T * c) @ U


def _check_pairs(S, cfg, U_or, th_or, k, tol_theta=1e-10):
    U = torch.zeros(k, cfg.nA, dtype=torch.float64, device="cuda")
    th = w.wc4d_get_ritz(S.ctx, U, k)
    assert np.allclose(th, th_or, rtol=tol_theta), (th[:4], th_or[:4])
    # sign-invariant comparison: C v for random vectors
    v = inputs.block(77, cfg.nA, 3)
    Cg, Co = _lmp_dense(host(U), th), _lmp_dense(U_or, th_or)
    assert np.abs(v @ Cg - v @ Co).max() < 1e-8 * np.abs(v).max()


@pytest.mark.parametrize("name", ["ad_direct", "ad_fft", "l96"])
@pytest.mark.parametrize("method", ["revd", "nystrom", "ritzit", "nystrom1"])
def test_sketch_fp64_matches_oracle(name, method):
    cfg, S, p, _ = setup(name)
    k, m = cfg.k, cfg.K
    G = inputs.probes(5, cfg.nA, m)
    w.wc4d_sketch(S.ctx, w.METHODS[method], k, m - k, cfg.q_power, 0, dev(G), w.FP64)
    Uo, tho = oracle_pairs(method, p, k, G, cfg.q_power)
    _check_pairs(S, cfg, Uo, tho, k)


def test_sketch_internal_probes_match_oracle_philox():
    cfg, S, p, _ = setup("ad_direct")
    k, m = cfg.k, cfg.K
    w.wc4d_sketch(S.ctx, w.REVD, k, m - k, 1, 2024, None, w.FP64)
    G = oracle.gaussian(2024, cfg.nA, m)
    Uo, tho = oracle.revd(p, k, G, q=1)
    _check_pairs(S, cfg, Uo, tho, k)


def test_products_with_A_per_method():
    cfg, S, _, _ = setup("ad_direct")
    for method, q, expect in (("revd", 0, 2), ("revd", 1, 3), ("nystrom", 0, 2), ("ritzit", 0, 1), ("nystrom1", 0, 1)):
        w.wc4d_hvp_count(S.ctx, reset=True)
        w.wc4d_sketch(S.ctx, w.METHODS[method], cfg.k, cfg.l, q, 3, None, w.FP64)
        assert w.wc4d_hvp_count(S.ctx) == expect, method


def test_lmp_apply_matches_oracle():
    cfg, S, p, _ = setup("ad_fft")
    G = inputs.probes(6, cfg.nA, cfg.K)
    Uo, tho = oracle.nystrom(p, cfg.k, G)
    w.wc4d_set_ritz(S.ctx, cfg.k, dev(Uo), tho)
    v = inputs.block(8, cfg.nA, 1)[0]
    y = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_lmp_apply(S.ctx, dev(v), y, 0)
    assert relerr(host(y), oracle.lmp_apply(Uo, tho, v)) < 1e-13
    w.wc4d_lmp_apply(S.ctx, dev(v), y, 1)
    assert relerr(host(y), oracle.lmp_apply(Uo, tho, v, transpose=True)) < 1e-13


# ------------------------------------------------------------------ PCG
@pytest.mark.parametrize("name", ["ad_direct", "ad_fft", "l96"])
@pytest.mark.parametrize("method", ["none", "revd", "nystrom", "ritzit", "nystrom1"])
def test_pcg_fp64_matches_oracle(name, method):
    """Same probes, same LMP construction, PCG from x_0 = 0.

    FP64 CG on these problems is itself chaotic after ~10 iterations: in the
    oracle alone a 1e-12 relative perturbation of the right-hand side moves
    iterate 20 by up to 3e-4 and iterate 35 by 1e-6, while the converged
    solution moves by only kappa * 1e-12.  Parity is therefore checked on
    (a) the first iterates, (b) the solution converged to 1e-12, and (c) at
    the working tolerance 1e-6: residual, iteration count and distance."""
    cfg, S, p, tw = setup(name)
    d = oracle.innovation(p, tw.xb, tw.y)
    b = oracle.rhs(p, d)
    k = cfg.k
    G = inputs.probes(11, cfg.nA, cfg.K)
    if method == "none":
        Uo = tho = None
        w.wc4d_set_ritz(S.ctx, 0, None, np.zeros(0))
        use = 0
    else:
        w.wc4d_sketch(S.ctx, w.METHODS[method], k, cfg.l, cfg.q_power, 0, dev(G), w.FP64)
        Uo, tho = oracle_pairs(method, p, k, G, cfg.q_power)
        use = 1
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    # (a) early iterates and their quadratic-cost decrease
    for it_f in (1, 4, 8):
        ro = oracle.pcg(p, b, Uo, tho, force_iters=it_f)
        it2, _, qcf2, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, use, it_f, w.FP64, qcf=True)
        assert it2 == it_f
        assert relerr(host(x), ro["x"]) < 1e-9, it_f
        assert np.allclose(qcf2, ro["qcf_drop"], rtol=1e-9)
    # (b) converged solution; without the LMP kappa(A) ~ 2.5e3 limits the
    # attainable accuracy of x to ~kappa * 1e-13
    ro = oracle.pcg(p, b, Uo, tho, tol=1e-13, maxit=5000)
    w.wc4d_pcg(S.ctx, x, 1e-13, 5000, use, 0, w.FP64, raise_on_noconv=False)
    assert relerr(host(x), ro["x"]) < (1e-10 if use else 5e-10)
    # (c) working tolerance
    ro = oracle.pcg(p, b, Uo, tho, tol=1e-6)
    it, rel, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, use, 0, w.FP64)
    # the count that first reaches 1e-6 agrees within 2, or within the
    # oracle's own plateau: where its residual lingers between 1e-6 and
    # 3e-6 (ritzit's curve does, for four iterations), rounding in the last
    # digits decides which iteration crosses
    hist = np.asarray(ro["relres_hist"][:ro["iters"]])
    plateau = int(np.sum(hist[-10:] <= 3e-6))
    assert rel <= 1e-6 and abs(it - ro["iters"]) <= max(2, plateau + 1), (it, ro["iters"], plateau)
    r = b - oracle.hvp(p, host(x)[None, :])[0]
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
    assert relerr(host(x), ro["x"]) < 1e-4


@pytest.mark.parametrize("name", ["ad_direct", "ad_fft", "l96"])
@pytest.mark.parametrize("method", ["revd", "nystrom", "ritzit", "nystrom1"])
def test_pcg_mixed_meets_tolerance(name, method):
    """Mixed path (FP32 sketch and CG, FP64 refinement): true relative
    residual <= 1e-6 at tol 1e-6 (checked with the oracle's own product) and,
    there, the distance to the oracle's solution that this residual allows
    (2e-6 |b|, since |A^{-1}| <= 1); the solution within 1e-5 of the oracle's
    when run to tol 1e-9 (at 1e-6 the relative distance of any two solvers'
    answers is bounded only by 2e-6 |b| / |x|, ~5e-4 on these windows)."""
    cfg, S, p, tw = setup(name)
    d = oracle.innovation(p, tw.xb, tw.y)
    b = oracle.rhs(p, d)
    xs = oracle.pcg(p, b, tol=1e-12, maxit=5000)["x"]
    w.wc4d_sketch(S.ctx, w.METHODS[method], cfg.k, cfg.l, cfg.q_power, 17, None, w.MIXED)
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, rel, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 1, 0, w.MIXED)
    assert rel <= 1e-6
    r = b - oracle.hvp(p, host(x)[None, :])[0]
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6
    # at the working tolerance: A = I + (positive semi-definite), so
    # |A^{-1}| <= 1 and every x with |b - A x| <= tol |b| is within tol |b|
    # of the exact solution; the mixed solution and the oracle's own PCG
    # solution at 1e-6 are therefore within (1.01 + 1) 1e-6 |b| of each other
    xo6 = oracle.pcg(p, b, tol=1e-6, maxit=5000)["x"]
    assert np.linalg.norm(host(x) - xo6) <= 2.01e-6 * np.linalg.norm(b)
    it, rel, _, _ = w.wc4d_pcg(S.ctx, x, 1e-9, 5000, 1, 0, w.MIXED)
    assert rel <= 1e-9
    assert relerr(host(x), xs) <= 1e-5


def test_inner_loop_entry_point():
    cfg, S, p, tw = setup("ad_direct")
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, rel = w.wc4d_inner_loop(S.ctx, w.REVD, cfg.k, cfg.l, cfg.q_power, 5, 1e-6, 5000, w.FP64, x)
    assert rel <= 1e-6 and it > 0
    d = oracle.innovation(p, tw.xb, tw.y)
    b = oracle.rhs(p, d)
    r = b - oracle.hvp(p, host(x)[None, :])[0]
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-6


# ------------------------------------------------------------------ edge cases and errors
def test_no_observations_gives_identity():
    cfg = inputs.scaled(inputs.TINY, n=32, N=2, k=3, l=2, obs_stride=4, obs_t0=9)
    tw = inputs.twin(cfg.replace(obs_t0=1))
    S = w.Solver(cfg)
    assert w.wc4d_nobs(S.ctx) == 0
    w.wc4d_set_background_obs(S.ctx, tw.xb, np.zeros(0))
    X = inputs.block(1, cfg.nA, 4)
    Y = torch.zeros(4, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X), Y, 4, cfg.nA)
    assert np.array_equal(host(Y), X)            # A = I exactly
    x = torch.ones(cfg.nA, dtype=torch.float64, device="cuda")
    it, rel, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 100, 0, 0, w.FP64)
    assert it == 0 and rel == 0.0 and float(x.abs().max()) == 0.0


def test_single_subwindow_and_odd_grid():
    cfg = inputs.scaled(inputs.TINY, n=99, N=1, k=3, l=2, obs_stride=7)
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    p = oracle_problem(cfg, xb=tw.xb)
    X = inputs.block(4, cfg.nA, 3)
    Y = torch.zeros(3, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X), Y, 3, cfg.nA)
    assert colrel(host(Y), oracle.hvp(p, X)) < 1e-12
    th = w.wc4d_sketch(S.ctx, w.RITZIT, 3, 2, 0, 1, None, w.FP64)
    _, tho = oracle.ritzit(p, 3, oracle.gaussian(1, cfg.nA, 5))
    assert np.allclose(th, tho, rtol=1e-10)


def test_invalid_arguments_are_rejected():
    cfg, S, _, _ = setup("ad_direct")
    bad = w.Problem()
    bad.n, bad.N, bad.sigma_o2, bad.obs_stride = 1, 5, 0.01, 1
    with pytest.raises(w.WC4DError):
        w.wc4d_create(bad)
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_hvp(S.ctx, x, x, 0, cfg.nA)
    assert e.value.status == w.EINVAL
    with pytest.raises(w.WC4DError):
        w.wc4d_sketch(S.ctx, w.REVD, 0, 1, 0, 0, None)
    fresh = w.Solver(cfg)              # no background / observations yet
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_pcg(fresh.ctx, x)
    assert e.value.status == w.ESTATE


def test_maxit_reports_no_convergence():
    cfg, S, _, _ = setup("ad_direct")
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, rel, _, st = w.wc4d_pcg(S.ctx, x, 1e-12, 2, 0, 0, w.FP64, raise_on_noconv=False)
    assert st == w.ENOCONV and it == 2 and rel > 1e-12


# ------------------------------------------------------------------ the benchmark's sketch width
@pytest.mark.parametrize("method", ["revd", "nystrom", "ritzit", "nystrom1"])
def test_sketch_256_columns_matches_oracle(method):
    """k + l = 256 (the width used on the large window): multi-tile, multi-split
    Gram products and a 256 x 256 one-sided Jacobi."""
    cfg = AD_FFT.replace(k=240, l=16)
    _, S, p, _ = setup("ad_fft")
    k, m = cfg.k, cfg.K
    G = inputs.probes(21, cfg.nA, m)
    w.wc4d_sketch(S.ctx, w.METHODS[method], k, m - k, cfg.q_power, 0, dev(G), w.FP64)
    Uo, tho = oracle_pairs(method, p, k, G, cfg.q_power)
    U = torch.zeros(k, cfg.nA, dtype=torch.float64, device="cuda")
    th = w.wc4d_get_ritz(S.ctx, U, k)
    # the top Ritz values are well separated; the tail of 240 values near 1 is not
    assert np.allclose(th[:40], tho[:40], rtol=1e-10)
    assert np.allclose(th, tho, rtol=1e-8, atol=1e-8)
    # mixed: the sweep products run as TF32 tensor-core MMAs (n = 128 is a
    # multiple of the 128-row tile), so the Ritz values carry ~1e-3 errors
    w.wc4d_sketch(S.ctx, w.METHODS[method], k, m - k, cfg.q_power, 0, dev(G), w.MIXED)
    th32 = w.wc4d_get_ritz(S.ctx, U, k)
    assert np.allclose(th32[:40], tho[:40], rtol=1e-2)


# ------------------------------------------------------------------ tensor-core sweeps
AD_TC = inputs.scaled(inputs.TINY, n=512, N=4, k=240, l=16, obs_stride=8)


@pytest.mark.parametrize("n,N,K", [(512, 4, 16), (512, 4, 48), (512, 4, 256), (1024, 3, 256), (2048, 3, 256),
                                   (4096, 2, 48), (4096, 2, 256)])
def test_tensor_core_sweeps_match_oracle(n, N, K):
    """Mixed sweeps with K a multiple of 16 and n a multiple of 128 run as
    tcgen05 TF32 MMAs, split-K over S CTAs per 128-row block with the
    partials summed in fixed order by a second kernel: S = 2 (n = 512), 4
    (n = 1024 and 4096, the large window's grid) and 8 (n = 2048).
    Operands are rounded to the nearest
    TF32 value (2^-11 relative, unbiased), so the error stays near 1e-4;
    the tensor cores' own truncation would bias every product by about
    -1e-3 and fail both checks."""
    cfg = AD_TC if n == 512 else inputs.scaled(inputs.TINY, n=n, N=N, k=240, l=16, obs_stride=8)
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    p = oracle_problem(cfg, xb=tw.xb)
    X = inputs.block(40 + K, cfg.nA, K)
    W = dev(X, torch.float32)
    w.wc4d_apply_linv(S.ctx, W, K, cfg.nA, w.MIXED)
    assert colrel(host(W), oracle.Linv(p, X)) < 1e-3
    Y = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, dev(X, torch.float32), Y, K, cfg.nA, w.MIXED)
    Ho = oracle.hvp(p, X)
    err = colrel(host(Y), Ho)
    assert err < 1e-3, err
    bias = np.mean(np.sum((host(Y) - Ho) * Ho, axis=1) / np.sum(Ho * Ho, axis=1))
    # measured: 9e-5 at n = 2048, 4.2e-4 at n = 4096 (the TF32 rounding of
    # the propagators; the FP32 products give -5e-7)
    assert abs(bias) < (6e-4 if n >= 4096 else 3e-4), bias
    S.close()


# ------------------------------------------------------------------ outer loop (Section 2.1)
def _forced_l96_traj(x0, eta, cfg):
    """All RK4 states of the forced Lorenz-96 run (eq. 1): eta_t is added at
    the end of subwindow t-1 (oracle primitives only)."""
    n, traj = cfg.n, [np.array(x0, dtype=np.float64)]
    x = traj[0].copy()
    for t in range(cfg.N):
        for k in range(cfg.steps):
            x = oracle.l96_rk4(x, cfg.F, cfg.dt)
            if k == cfg.steps - 1:
                x = x + eta[(t + 1) * n:(t + 2) * n]
            traj.append(x.copy())
    return np.array(traj)


@pytest.mark.parametrize("name", ["ad_direct", "ad_fft", "l96"])
def test_outer_update_matches_oracle(name):
    """Two outer-loop updates (eq. 3): p += D^{1/2} x, D^{-1/2} b -= x, model
    re-run with forcing, innovations and rhs; compared with the oracle's
    forward run with forcing, innovations and rhs, and (Lorenz-96) the
    Hessian product along the new trajectory."""
    cfg = CASES[name]
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    p = oracle_problem(cfg, mode="stepping", xb=tw.xb)
    n, nA = cfg.n, cfg.nA
    x0, eta, Dm12b = tw.xb.copy(), np.zeros(nA), np.zeros(nA)
    for j, scale in enumerate((0.05, 0.02)):
        x = scale * inputs.block(300 + j, nA, 1)[0]
        w.wc4d_outer_update(S.ctx, dev(x))
        dp = oracle.Dsqrt(p, x[None, :])[0]
        x0 = x0 + dp[:n]
        eta[n:] += dp[n:]
        Dm12b -= x
        if cfg.model == inputs.MODEL_L96:
            bs, qs = p.Bsqrt, p.Qsqrt
            p = oracle.Problem(model=oracle.MODEL_L96, F=cfg.F, traj=_forced_l96_traj(x0, eta, cfg), n=n, N=cfg.N,
                               Bsqrt=bs, Qsqrt=qs, sigma_o2=cfg.sigma_o2, obs_stride=cfg.obs_stride,
                               obs_t0=cfg.obs_t0, steps=cfg.steps, dt=cfg.dt)
        d = oracle.innovation(p, x0, tw.y, eta)
        r = oracle.rhs(p, d, Dm12b)
        got = torch.zeros(nA, dtype=torch.float64, device="cuda")
        w.wc4d_get_rhs(S.ctx, got)
        assert relerr(host(got), r) < 1e-10, (j, relerr(host(got), r))
    if cfg.model == inputs.MODEL_L96:
        X = inputs.block(310, nA, 3)
        Y = torch.zeros(3, nA, dtype=torch.float64, device="cuda")
        w.wc4d_hvp(S.ctx, dev(X), Y, 3, nA, w.FP64)
        assert colrel(host(Y), oracle.hvp(p, X)) < 1e-11
    S.close()


@pytest.mark.parametrize("name", ["ad_fft", "l96"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_graph_replay_is_bitwise_eager(name, precision):
    """The CG iterations run from captured CUDA graphs -- the device-side
    WHILE loop and one graph launch per iteration -- compute exactly what the
    eager launches compute: same iterates, counts and QCF history.  The
    solver's stream is the legacy default stream, which cannot be captured:
    the graphs must still engage (captured on the context's own stream)."""
    cfg, S, p, tw = setup(name)
    prec = w.FP64 if precision == "fp64" else w.MIXED
    w.wc4d_sketch(S.ctx, w.REVD, cfg.k, cfg.l, cfg.q_power, 41, None, prec)
    out = []
    for graphs, mode in ((0, w.ITER_EAGER), (1, w.ITER_DEVICE_LOOP), (2, w.ITER_GRAPH_PER_ITERATION)):
        w.wc4d_set_graphs(S.ctx, graphs)
        x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
        it, rel, qcf, _ = w.wc4d_pcg(S.ctx, x, 1e-9, 5000, 1, 0, prec, qcf=True)
        assert w.wc4d_iteration_mode(S.ctx) == (mode, ""), (graphs, w.wc4d_iteration_mode(S.ctx))
        out.append((it, rel, host(x), np.asarray(qcf)))
    w.wc4d_set_graphs(S.ctx, True)
    i0, r0, x0, q0 = out[0]
    assert i0 > 2
    for i1, r1, x1, q1 in out[1:]:
        assert i0 == i1
        assert r0 == r1
        assert np.array_equal(x0, x1)
        assert np.array_equal(q0, q1)
