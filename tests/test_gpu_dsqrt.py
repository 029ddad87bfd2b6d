"""D^{1/2} (the block-diagonal covariance square root of eq. 10, circulant
B^{1/2} and Q^{1/2} on the periodic grid) at the grid sizes of the large
windows, where the on-chip Stockham FFT runs (n = 512 .. 8192: radix-16
passes plus one radix-2, 4 or 8 pass), for one column, an odd column count
(the last complex transform carries one real vector) and a block, in FP64
and FP32, against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

_cache = {}


def setup(n, N):
    key = (n, N)
    if key not in _cache:
        cfg = inputs.scaled(inputs.LARGE, n=n, N=N, k=8, l=4)
        S = w.Solver(cfg, M_shared=True)
        p = oracle_problem(cfg, mode="stepping")
        _cache[key] = (cfg, S, p)
    return _cache[key]


def colrel(A, B):
    return max(np.linalg.norm(A[j] - B[j]) / np.linalg.norm(B[j]) for j in range(B.shape[0]))


@pytest.mark.parametrize("n,N", [(512, 3), (1024, 2), (2048, 3), (4096, 2), (8192, 2)])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_dsqrt_stockham_matches_oracle(n, N, K):
    cfg, S, p = setup(n, N)
    X = inputs.block(500 + n + K, cfg.nA, K)
    ref = oracle.Dsqrt(p, X)
    Y = torch.zeros(K, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, torch.as_tensor(X, device="cuda"), Y, K, cfg.nA)
    # FP64: both sides take the square-root spectrum from their own O(n)
    # DFT sums of the covariance row (eigenvalue errors ~eps n lambda_max,
    # amplified in the square roots of the smallest eigenvalues): ~1e-12
    # relative at n = 2048
    assert colrel(Y.cpu().numpy(), ref) < 1e-11
    Y32 = torch.zeros(K, cfg.nA, dtype=torch.float32, device="cuda")
    w.wc4d_apply_dsqrt(S.ctx, torch.as_tensor(X, dtype=torch.float32, device="cuda"), Y32, K, cfg.nA, w.MIXED)
    # FP32: rounding of x, of the two transforms and of y
    assert colrel(Y32.double().cpu().numpy(), ref) < 1e-5
