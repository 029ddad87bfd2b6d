"""Ritz pairs from CG (Section 3.3, eq. 18-20) on the GPU against the oracle:
the tridiagonal T_J built from CG's alpha_j, beta_j, its leading eigenpairs
and the Ritz vectors u_i = F_J w_i, and the deterministic LMP they give."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

CASES = {"ad_direct": inputs.TINY,
         "ad_fft": inputs.scaled(inputs.TINY, n=128, N=6, k=12, l=4, obs_stride=6)}
_cache = {}


def setup(name):
    if name not in _cache:
        cfg = CASES[name]
        tw = inputs.twin(cfg)
        S = w.Solver(cfg, tw)
        p = oracle_problem(cfg, mode="stepping", xb=tw.xb)
        b = oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))
        _cache[name] = (cfg, S, p, b)
    return _cache[name]


def _lmp_dense(U, th):
    c = 1.0 - 1.0 / np.sqrt(th)
    return np.eye(U.shape[1]) - (U.T * c) @ U


@pytest.mark.parametrize("name", list(CASES))
def test_tridiagonal_matches_oracle(name):
    """First iterations (before rounding makes the two CGs drift apart):
    gamma and tau of T_J agree to ~1e-11."""
    cfg, S, p, b = setup(name)
    J = 8
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, _ = w.wc4d_lanczos_cg(S.ctx, x, 0.0, J, reorth=True)
    assert it == J
    g, t = w.wc4d_lanczos_tridiag(S.ctx, J)
    out = oracle.lanczos_cg(p, b, J, reorth=True)
    To = oracle.lanczos_tridiag(out["alpha"], out["beta"])
    assert np.allclose(g, np.diag(To), rtol=1e-10)
    assert np.allclose(t, np.diag(To, 1), rtol=1e-10)
    assert np.linalg.norm(x.cpu().numpy() - out["x"]) <= 1e-10 * np.linalg.norm(out["x"])


@pytest.mark.parametrize("name", list(CASES))
def test_ritz_pairs_match_oracle_and_precondition(name):
    """Converged leading Ritz pairs after 40 reorthogonalised iterations agree
    with the oracle's, and installed as the LMP they cut the CG iterations of
    the next solve (the deterministic LMP of Section 3.3)."""
    cfg, S, p, b = setup(name)
    J, k = 40, 5
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_lanczos_cg(S.ctx, x, 0.0, J, reorth=True)
    th = w.wc4d_lanczos_ritz(S.ctx, k)
    out = oracle.lanczos_cg(p, b, J, reorth=True)
    Uo, tho = oracle.lanczos_ritz(out["alpha"], out["beta"], out["F"], k)
    assert np.allclose(th, tho, rtol=1e-8)
    U = torch.zeros(k, cfg.nA, dtype=torch.float64, device="cuda")
    th2 = w.wc4d_get_ritz(S.ctx, U, k)
    assert np.array_equal(th2, th)
    v = inputs.block(77, cfg.nA, 3)
    Cg, Co = _lmp_dense(U.cpu().numpy(), th), _lmp_dense(Uo, tho)
    assert np.abs(v @ Cg - v @ Co).max() < 1e-6 * np.abs(v).max()
    # the deterministic LMP in the next solve
    it_lmp, rel_lmp, _, _ = w.wc4d_pcg(S.ctx, x, 1e-8, 5000, 1, 0, w.FP64)
    it_none, rel_none, _, _ = w.wc4d_pcg(S.ctx, x, 1e-8, 5000, 0, 0, w.FP64)
    assert rel_lmp <= 1e-8 and rel_none <= 1e-8
    assert it_lmp < it_none


def test_without_reorthogonalisation_values_stay_in_the_spectrum():
    cfg, S, p, b = setup("ad_direct")
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it, _ = w.wc4d_lanczos_cg(S.ctx, x, 1e-10, 300, reorth=False)
    th = w.wc4d_lanczos_ritz(S.ctx, 8)
    from problems import dense_A
    A = dense_A(p)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert np.all(th <= lam[-1] * (1 + 1e-8)) and np.all(th >= lam[0] * (1 - 1e-8))
    assert abs(th[0] - lam[-1]) <= 1e-8 * lam[-1]


def test_lanczos_state_errors():
    cfg = inputs.TINY
    S = w.Solver(cfg, inputs.twin(cfg))
    with pytest.raises(w.WC4DError):
        w.wc4d_lanczos_ritz(S.ctx, 3)            # no Lanczos data yet
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_lanczos_cg(S.ctx, x, 0.0, 4)
    with pytest.raises(w.WC4DError):
        w.wc4d_lanczos_ritz(S.ctx, 5)            # k > J
    S.close()
