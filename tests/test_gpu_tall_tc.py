"""The CholeskyQR product Y R^{-1} of the mixed sketch on the tensor cores
(3xTF32: Y and R^{-1} split into TF32 values and remainders, three products
summed in FP32 tensor memory), through the C-ABI (wc4d_orthonormalize with
FP32 blocks), against the FP32-pipe product: after CholeskyQR2 both return
columns orthonormal to FP32 rounding with Y = Z R, on ragged row counts,
leading dimensions that are not multiples of 4, m = 64 .. 256 and
condition numbers up to 1e5, and give the same R to FP32 accuracy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
from paper_2101_07249_gb300 import inputs

pytestmark = pytest.mark.gpu


def _orthonormalize(S, A32, ld, tc):
    rows, m = A32.shape
    Yd = torch.zeros(m * ld, dtype=torch.float32, device="cuda")
    Yd.view(m, ld)[:, :rows] = torch.as_tensor(A32.T.astype(np.float32))
    w.wc4d_set_gram_path(S.ctx, tc)
    R = w.wc4d_orthonormalize(S.ctx, Yd, rows, m, ld, precision=w.MIXED)
    w.wc4d_set_gram_path(S.ctx, True)
    Z = Yd.view(m, ld)[:, :rows].double().cpu().numpy().T
    return Z, R


@pytest.mark.parametrize("m,rows,ld,cond", [(256, 70001, 70003, 1e3), (128, 20000, 20001, 1e5),
                                            (64, 131, 135, 10.0)])
def test_cholqr2_tensor_core_product_matches_fp32_pipe(m, rows, ld, cond):
    S = w.Solver(inputs.TINY, inputs.twin(inputs.TINY))
    g = np.random.default_rng(m + rows)
    Q1, _ = np.linalg.qr(g.standard_normal((rows, m)))
    V, _ = np.linalg.qr(g.standard_normal((m, m)))
    A32 = ((Q1 * np.logspace(0, -np.log10(cond), m)) @ V.T).astype(np.float32).astype(np.float64)
    out = {}
    for tc in (True, False):
        Z, R = _orthonormalize(S, A32, ld, tc)
        assert np.abs(Z.T @ Z - np.eye(m)).max() < 2e-5, tc
        assert np.linalg.norm(A32 - Z @ R) / np.linalg.norm(A32) < 1e-5, tc
        assert np.all(np.diag(R) > 0)
        out[tc] = R
    assert np.abs(out[True] - out[False]).max() < 1e-5 * np.abs(out[False]).max()
    S.close()
