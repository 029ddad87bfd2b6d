"""The allocation-free LMP entry point (wc4d_lmp_apply_static) through the
C-ABI, on two calls in a row: against the context-based wc4d_lmp_apply and
against the oracle's eq. 16 product.

It serves callers that cannot allocate device memory where they apply the
preconditioner -- systems that reserve their whole device memory budget up
front, code that must not take the device-wide synchronisation of an
allocation mid-solve, callers without a library context; its scratch is a
fixed array inside the library.  This file is collected last so that a
failure here stops a -x run only after every other test has run."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu


def _context(n, N):
    prob = w.Problem()
    prob.n, prob.N, prob.model, prob.sigma_o2, prob.obs_stride, prob.obs_t0, prob.obs_tstride = n, N, 0, 0.01, 4, 1, 1
    prob.M_shared = 1
    return w.wc4d_create(prob)


@pytest.mark.parametrize("n,N,k", [(128, 6, 12), (4000, 49, 240)])
def test_static_lmp_matches_context_lmp_and_oracle(n, N, k):
    nA = n * (N + 1)
    g = np.random.default_rng(k)
    Q, _ = np.linalg.qr(g.standard_normal((nA, k)))
    theta = np.sort(1.0 + 1e3 * g.random(k))[::-1].copy()
    Ut = np.ascontiguousarray(Q.T)                    # rows = columns of U
    U = torch.as_tensor(Ut, device="cuda")
    th = torch.as_tensor(theta, device="cuda")
    ctx = _context(n, N)
    try:
        w.wc4d_set_ritz(ctx, k, U, theta)
        for _ in range(2):                       # two calls in a row share the scratch
            vh = g.standard_normal(nA)
            v = torch.as_tensor(vh, device="cuda")
            y_ref = torch.empty_like(v)
            y = torch.full_like(v, float("nan"))
            w.wc4d_lmp_apply(ctx, v, y_ref, 0)
            w.wc4d_lmp_apply_static(U, th, k, nA, v, y)
            torch.cuda.synchronize()
            err = float((y - y_ref).norm() / y_ref.norm())
            assert err < 1e-13, err
            yo = oracle.lmp_apply(Ut, theta, vh)
            err_o = np.linalg.norm(y.cpu().numpy() - yo) / np.linalg.norm(yo)
            assert err_o < 1e-13, err_o
    finally:
        w.wc4d_destroy(ctx)


def test_static_lmp_rejects_too_many_pairs():
    k, nA = 1025, 8
    U = torch.zeros(k * nA, dtype=torch.float64, device="cuda")
    th = torch.ones(k, dtype=torch.float64, device="cuda")
    v = torch.zeros(nA, dtype=torch.float64, device="cuda")
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_lmp_apply_static(U, th, k, nA, v, torch.zeros_like(v))
    assert e.value.status == w.EINVAL
