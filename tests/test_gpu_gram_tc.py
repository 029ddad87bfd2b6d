"""FP64-accurate Gram-type products of FP32 blocks on the tensor cores
(sliced BF16 operands, exact FP32 chunk sums in tensor memory) against the
exact FP64 product of the same FP32 data, and against the FP32-pipe
double-float kernel, through the C-ABI (wc4d_gram_sym).  Cases: ragged row
counts (a partial 64-row block, a partial 512-row chunk, a split with no
rows left), m = 128 and 256, columns whose scales span 2^+-20, an ill-
conditioned block (kappa = 1e5), a zero column, two distinct operands (the
Rayleigh-Ritz form Z^T E, upper tiles), and shapes that take the FP32-pipe
path (m not a multiple of 128, fewer than 512 rows)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
from paper_2101_07249_gb300 import inputs

pytestmark = pytest.mark.gpu


def _ctx():
    cfg = inputs.TINY
    return w.Solver(cfg, inputs.twin(cfg))


def _gram(S, Y, E=None, tc=True):
    m, rows = Y.shape
    w.wc4d_set_gram_path(S.ctx, tc)
    A = torch.as_tensor(np.ascontiguousarray(Y, dtype=np.float32), device="cuda")
    B = A if E is None else torch.as_tensor(np.ascontiguousarray(E, dtype=np.float32), device="cuda")
    C = torch.empty(m * m, dtype=torch.float64, device="cuda")
    w.wc4d_gram_sym(S.ctx, A, rows, B, rows, rows, m, C, w.MIXED)
    w.wc4d_set_gram_path(S.ctx, True)
    return C.cpu().numpy().reshape(m, m).T      # column-major -> C[i, j]


def _exact(Y, E=None):
    Y64 = Y.astype(np.float32).astype(np.float64)
    E64 = Y64 if E is None else E.astype(np.float32).astype(np.float64)
    return Y64 @ E64.T


def _scaled_err(G, ref, Y, E=None):
    """max |G - ref| / (|y_i| |e_j|): the error relative to the Cauchy-Schwarz bound of each entry."""
    ny = np.linalg.norm(Y.astype(np.float64), axis=1)
    ne = ny if E is None else np.linalg.norm(E.astype(np.float64), axis=1)
    den = np.outer(ny, ne)
    den[den == 0] = 1.0
    return np.max(np.abs(G - ref) / den)


@pytest.mark.parametrize("m,rows", [(128, 5000), (128, 4096 + 64 * 9 + 7), (256, 70001), (256, 167936)])
def test_gram_tc_matches_exact_product(m, rows):
    S = _ctx()
    g = np.random.default_rng(m + rows)
    Y = g.standard_normal((m, rows)).astype(np.float32)
    ref = _exact(Y)
    G = _gram(S, Y)
    # slices keep 41 bits below each column's largest entry: the error of an
    # entry is a few 2^-41 max|y_i| max|y_j| per row, summed with random signs
    assert _scaled_err(G, ref, Y) < 2e-11
    assert np.array_equal(G, G.T)                 # mirrored
    Gdf = _gram(S, Y, tc=False)
    # double-float sums per row split: ~2^-46 per term, 2.5e-13 measured at 167 936 rows
    assert _scaled_err(Gdf, ref, Y) < 1e-12
    S.close()


def test_gram_tc_wide_scales_ill_conditioned_and_zero_column():
    S = _ctx()
    g = np.random.default_rng(7)
    m, rows = 256, 20000 + 33
    U, _ = np.linalg.qr(g.standard_normal((rows, m)))
    V, _ = np.linalg.qr(g.standard_normal((m, m)))
    Y = ((U * np.logspace(0, -5, m)) @ V.T).T                  # kappa = 1e5
    Y *= np.exp2(g.integers(-20, 21, m))[:, None]              # column scales 2^-20 .. 2^20
    Y[17] = 0.0
    Y = Y.astype(np.float32)
    ref = _exact(Y)
    G = _gram(S, Y)
    assert _scaled_err(G, ref, Y) < 2e-11
    assert np.all(G[17] == 0) and np.all(G[:, 17] == 0)
    # the Cholesky factor of the tensor-core Gram: G + dG with |dG| ~ 1e-12 |G|
    # against kappa(G) = 1e10 -- still positive definite, as CholeskyQR needs
    keep = np.ones(m, bool)
    keep[17] = False
    np.linalg.cholesky(G[np.ix_(keep, keep)])
    S.close()


def test_gram_tc_two_operands_upper_tiles():
    S = _ctx()
    g = np.random.default_rng(11)
    m, rows = 256, 33333
    Z = g.standard_normal((m, rows)).astype(np.float32)
    E = (g.standard_normal((m, rows)) * 3.0).astype(np.float32)
    ref = _exact(Z, E)
    G = _gram(S, Z, E)
    up = np.add.outer(np.arange(m) // 64, -(np.arange(m) // 64)) <= 0   # tiles i/64 <= j/64 are computed
    err = np.abs(G - ref) / np.outer(np.linalg.norm(Z.astype(np.float64), axis=1),
                                     np.linalg.norm(E.astype(np.float64), axis=1))
    assert np.max(err[up]) < 2e-11
    S.close()


@pytest.mark.parametrize("m,rows", [(64, 5000), (192, 3000), (128, 400)])
def test_gram_shapes_outside_the_tensor_core_path(m, rows):
    S = _ctx()
    Y = np.random.default_rng(m).standard_normal((m, rows)).astype(np.float32)
    G = _gram(S, Y)
    assert _scaled_err(G, _exact(Y), Y) < 1e-12            # the FP32-pipe double-float kernel
    S.close()
