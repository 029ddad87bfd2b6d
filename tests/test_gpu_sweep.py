"""The one-column sweeps of L^{-1} and L^{-T} (eq. 5 and its transpose, the
PCG matvec) at the grid sizes of the large windows: FP32 at n = 2048 and
4096 (the staged persistent kernel, n a multiple of 512 sixteen-byte
vectors), FP64 at n = 1024, 2048 and 4096, with one propagator shared by all
subwindows and with one stored per subwindow, against the FP64 oracle on the
same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

_cache = {}


def setup(n, N, shared):
    key = (n, N, shared)
    if key not in _cache:
        cfg = inputs.scaled(inputs.LARGE, n=n, N=N, k=8, l=4)
        S = w.Solver(cfg, M_shared=shared)
        p = oracle_problem(cfg, mode="dense")
        _cache[key] = (cfg, S, p)
    return _cache[key]


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


def sweeps(S, cfg, X, precision):
    dt = torch.float64 if precision == w.FP64 else torch.float32
    out = []
    for fn in (w.wc4d_apply_linv, w.wc4d_apply_linvT):
        Wd = torch.as_tensor(X, dtype=dt, device="cuda").contiguous()
        fn(S.ctx, Wd, 1, cfg.nA, precision)
        out.append(Wd.double().cpu().numpy())
    return out


@pytest.mark.parametrize("n,N", [(1024, 5), (2048, 3), (4096, 4)])
@pytest.mark.parametrize("shared", [True, False])
def test_staged_sweep_fp64_matches_oracle(n, N, shared):
    cfg, S, p = setup(n, N, shared)
    X = inputs.block(70 + n, cfg.nA, 1)
    fwd, adj = sweeps(S, cfg, X, w.FP64)
    assert colrel(fwd, oracle.Linv(p, X)) < 1e-12
    assert colrel(adj, oracle.LinvT(p, X)) < 1e-12


@pytest.mark.parametrize("n,N", [(2048, 3), (4096, 4)])
@pytest.mark.parametrize("shared", [True, False])
def test_staged_sweep_fp32_matches_oracle(n, N, shared):
    cfg, S, p = setup(n, N, shared)
    X = inputs.block(90 + n, cfg.nA, 1)
    fwd, adj = sweeps(S, cfg, X, w.MIXED)
    assert colrel(fwd, oracle.Linv(p, X)) < 1e-5
    assert colrel(adj, oracle.LinvT(p, X)) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_and_per_subwindow_propagators_agree_bitwise(precision):
    prec = w.FP64 if precision == "fp64" else w.MIXED
    cfg, S1, _ = setup(2048, 3, True)
    _, S2, _ = setup(2048, 3, False)
    X = inputs.block(123, cfg.nA, 1)
    a = sweeps(S1, cfg, X, prec)
    b = sweeps(S2, cfg, X, prec)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_staged_sweep_repeatable():
    cfg, S, _ = setup(4096, 4, False)
    X = inputs.block(7, cfg.nA, 1)
    a = sweeps(S, cfg, X, w.MIXED)
    b = sweeps(S, cfg, X, w.MIXED)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_autotuned_sweep_gemm_matches_oracle():
    """A block product whose propagator GEMMs take the SIMT path (K = 40 is
    not a multiple of 16): the first product tunes the tile shape of the
    (n, K, n) GEMM, every later product reuses it, and the results match the
    oracle to FP32 rounding whichever tile won."""
    n, N, K = 512, 3, 40
    cfg = inputs.scaled(inputs.LARGE, n=n, N=N, k=8, l=4)
    S = w.Solver(cfg, M_shared=True)
    p = oracle_problem(cfg, mode="dense")
    X = inputs.block(321, cfg.nA, K)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y, K, cfg.nA, w.MIXED)
    choice = w.wc4d_autotune_choice(False, n, K, n)
    assert 0 <= choice < 5
    assert colrel(Y.double().cpu().numpy(), oracle.hvp(p, X)) < 2e-5
    Y2 = torch.zeros_like(Y)
    w.wc4d_hvp(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y2, K, cfg.nA, w.MIXED)
    assert torch.equal(Y, Y2)                        # the cached tile: same launches, same bits
    assert w.wc4d_autotune_choice(False, n, K, n) == choice
    S.close()
