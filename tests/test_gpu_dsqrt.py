"""D^{1/2} (the block-diagonal covariance square root of eq. 10, circulant
B^{1/2} and Q^{1/2} on the periodic grid) at the grid sizes of the large
windows, where the on-chip Stockham FFT runs (n = 512 .. 8192: radix-16
passes plus one radix-2, 4 or 8 pass), for one column, an odd column count
(the last complex transform carries one real vector) and a block, in FP64
and FP32, against the FP64 oracle on the same seeded inputs: SOAR
covariances (the advection-diffusion windows) and the Gaussian B with the
identity Q of the Lorenz-96 window, whose spectrum falls to ~1e-34 of its
largest value at the shortest waves."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

_cache = {}


def setup(n, N, gauss=False):
    key = (n, N, gauss)
    if key not in _cache:
        cfg = inputs.scaled(inputs.LARGE, n=n, N=N, k=8, l=4)
        if gauss == "bdiag":    # B a multiple of the identity, Q SOAR (no transform of block 0)
            cfg = cfg.replace(b_kind=inputs.DIAG, b_var=0.3)
        elif gauss:     # the Lorenz-96 covariances on the advection-diffusion model (no transform of Q's blocks)
            L96 = inputs.L96
            cfg = cfg.replace(b_kind=L96.b_kind, b_var=L96.b_var, b_L=L96.b_L, q_kind=L96.q_kind,
                              q_var=L96.q_var, q_L=L96.q_L)
        S = w.Solver(cfg, M_shared=True)
        p = oracle_problem(cfg, mode="stepping")
        _cache[key] = (cfg, S, p)
    return _cache[key]


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


@pytest.mark.parametrize("n,N,gauss", [(512, 3, False), (1024, 2, False), (2048, 3, False), (4096, 2, False),
                                       (8192, 2, False), (1024, 2, True), (8192, 2, True), (2048, 3, "bdiag")])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_dsqrt_stockham_matches_oracle(n, N, gauss, K):
    cfg, S, p = setup(n, N, gauss)
    X = inputs.block(500 + n + K, cfg.nA, K)
    ref = oracle.Dsqrt(p, X)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, torch.as_tensor(X, device="cuda"), Y, K, cfg.nA)
    # FP64: the oracle's square-root spectrum is exact to double rounding
    # (extended-precision DFT of the SOAR row; Poisson closed form of the
    # Gaussian).  The library's SOAR closed form sums powers of the rounded
    # a = e^{-1/L}: the longest-wave eigenvalues (sum_r (1 + r/L) a^r, mean
    # power ~3L) carry a relative error of ~3 L eps, 5e-14 at L = 164 (n =
    # 8192), half of it in the root; each FP64 transform adds ~eps log2 n.
    # Measured: 2.4e-13 at n = 8192, K = 1.
    assert colrel(Y.cpu().numpy(), ref) < 5e-13
    Y32 = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, K, cfg.nA, w.MIXED)
    # FP32: rounding of x, of the two transforms and of y
    assert colrel(Y32.double().cpu().numpy(), ref) < 1e-5
