"""Host-visible failure statuses for non-finite inputs, injected on the host
(a NaN in one probe column, a NaN observation), and for bounded device-side
waits that run out (a wait limit of 0): the library must return an error
status -- not trap, hang or report success -- and the context must stay
usable, giving the same results afterwards as before the fault."""
import numpy as np
import pytest

from paper_2101_07249_gb300 import inputs

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu


def _solver():
    cfg = inputs.TINY
    tw = inputs.twin(cfg)
    return cfg, tw, w.Solver(cfg, tw)


def test_nan_probe_column_is_reported_and_the_context_recovers():
    cfg, tw, S = _solver()
    m = cfg.k + cfg.l
    G = inputs.probes(5, cfg.nA, m)
    th0 = w.wc4d_sketch(S.ctx, w.REVD, cfg.k, cfg.l, cfg.q_power, 0,
                        torch.as_tensor(G, device="cuda"), w.FP64)
    Gbad = G.copy()
    Gbad[3, 17] = np.nan                       # one entry of probe column 3
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_sketch(S.ctx, w.REVD, cfg.k, cfg.l, cfg.q_power, 0, torch.as_tensor(Gbad, device="cuda"), w.FP64)
    assert e.value.status in (w.ENOTSPD, w.ENAN, w.EBREAKDOWN)
    th1 = w.wc4d_sketch(S.ctx, w.REVD, cfg.k, cfg.l, cfg.q_power, 0,
                        torch.as_tensor(G, device="cuda"), w.FP64)
    assert np.allclose(th1, th0, rtol=1e-12, atol=0)
    S.close()


def test_nan_observation_is_reported_and_the_context_recovers():
    cfg, tw, S = _solver()
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it0, rel0, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 0, w.FP64)
    ybad = np.array(tw.y, dtype=np.float64).copy()
    ybad[7] = np.nan
    w.wc4d_set_background_obs(S.ctx, tw.xb, ybad)
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 0, w.FP64)
    assert e.value.status in (w.EBREAKDOWN, w.ENAN)
    w.wc4d_set_background_obs(S.ctx, tw.xb, tw.y)
    it1, rel1, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 0, w.FP64)
    assert it1 == it0 and rel1 <= 1e-6 and abs(rel1 - rel0) <= 1e-12
    S.close()


def test_grid_barrier_timeout_is_reported_and_the_context_recovers():
    """A bounded device-side wait that runs out: with a wait limit of 0 the
    persistent FP64 sweep's grid barrier gives up at its first incomplete
    poll (no asynchronous copy is in flight there), the kernel records the
    failure and returns, and the solve returns WC4D_ETIMEOUT; with the
    default limit restored the context reproduces its earlier result
    bit for bit."""
    cfg, tw, S = _solver()
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it0, rel0, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 8, w.FP64)
    x0 = x.cpu().numpy().copy()
    w.wc4d_set_wait_limit(S.ctx, 0)
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 8, w.FP64)
    assert e.value.status == w.ETIMEOUT
    w.wc4d_set_wait_limit(S.ctx, -1)
    x.zero_()
    it1, rel1, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5000, 0, 8, w.FP64)
    assert it1 == it0 == 8 and rel1 == rel0
    assert np.array_equal(x.cpu().numpy(), x0)
    S.close()


def test_l96_staged_copy_timeout_is_reported_and_the_context_recovers():
    """The FP32 Lorenz-96 sweeps wait, bounded, on the bulk copies that stage
    the trajectory's stage states.  With a wait limit of 0 every such wait
    gives up at once: the sweep's threads leave together, thread 0 first
    waits for the copies still in flight, and the product (one column, and a
    block with two columns per CTA; reported by wc4d_sync, as the product
    call itself does not synchronise) and a mixed PCG solve return
    WC4D_ETIMEOUT.  With the default limit restored the context reproduces
    its earlier results bit for bit."""
    cfg = inputs.L96.replace(name="l96_n256_N2", n=256, N=2, steps=4)
    S = w.Solver(cfg, inputs.twin(cfg, spinup=5.0))
    for K in (1, 70):
        X = torch.as_tensor(inputs.block(1200 + K, cfg.nA, K), dtype=torch.float32, device="cuda")
        Y0 = torch.zeros_like(X)
        w.wc4d_hvp(S.ctx, X, Y0, K, cfg.nA, w.MIXED)
        w.wc4d_set_wait_limit(S.ctx, 0)
        w.wc4d_hvp(S.ctx, X, torch.zeros_like(X), K, cfg.nA, w.MIXED)    # queued; the failure surfaces at the sync
        with pytest.raises(w.WC4DError) as e:
            w.wc4d_sync(S.ctx)
        assert e.value.status == w.ETIMEOUT
        w.wc4d_set_wait_limit(S.ctx, -1)
        Y1 = torch.zeros_like(X)
        w.wc4d_hvp(S.ctx, X, Y1, K, cfg.nA, w.MIXED)
        assert torch.equal(Y1, Y0)
    x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
    it0, rel0, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5, 0, 5, w.MIXED, raise_on_noconv=False)
    x0 = x.cpu().numpy().copy()
    w.wc4d_set_wait_limit(S.ctx, 0)
    x.zero_()
    with pytest.raises(w.WC4DError) as e:
        w.wc4d_pcg(S.ctx, x, 1e-6, 5, 0, 5, w.MIXED, raise_on_noconv=False)
    assert e.value.status == w.ETIMEOUT
    w.wc4d_set_wait_limit(S.ctx, -1)
    x.zero_()
    it1, rel1, _, _ = w.wc4d_pcg(S.ctx, x, 1e-6, 5, 0, 5, w.MIXED, raise_on_noconv=False)
    assert it1 == it0 and rel1 == rel0
    assert np.array_equal(x.cpu().numpy(), x0)
    S.close()
