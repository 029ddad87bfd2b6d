"""The learned-probe network on the device against the oracle's numpy FP64
version (BF16 weights, FP32 sums on the device), on a small Lorenz-96
window, and the learned start block through the randomised range finder."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu

L96S = inputs.L96.replace(name="l96_n64_N4", n=64, N=4, steps=3, obs_stride=4, k=8, l=4)


def random_net(N, m, seed):
    g = np.random.default_rng(seed)
    shapes = [(64, 2 * (N + 1), 5), (64, 64, 5), (64, 64, 5), (m * (N + 1), 64, 1)]
    Ws = [g.standard_normal(s) / np.sqrt(s[1] * s[2]) for s in shapes]
    bits = [(W.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16) for W in Ws]   # truncate to BF16
    bs = [0.1 * g.standard_normal(s[0]).astype(np.float32) for s in shapes]
    return bits, bs


def test_learned_probes_match_oracle():
    cfg, m = L96S, 6
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw)
    bits, bs = random_net(cfg.N, m, 5)
    wdev = torch.as_tensor(np.concatenate([b.ravel() for b in bits]).view(np.int16), device="cuda")
    bdev = torch.as_tensor(np.concatenate(bs), device="cuda")
    out = torch.zeros(m, cfg.nA, dtype=torch.float64, device="cuda")
    w.wc4d_learned_probes(S.ctx, wdev, bdev, m, out, cfg.nA)
    traj = oracle.l96_run(tw.xb, cfg.F, cfg.dt, cfg.N * cfg.steps)[::cfg.steps]
    mask = np.zeros((cfg.N + 1, cfg.n))
    for t in range(cfg.obs_t0, cfg.N + 1):
        mask[t, ::cfg.obs_stride] = 1.0
    Ws = [oracle.bf16_to_f64(b) for b in bits]
    ref = oracle.learned_probes(traj, cfg.F, mask, Ws, [b.astype(np.float64) for b in bs], m)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    # the learned block through Alg. 3: an explicit probe block [S, G]
    G = np.concatenate([ref, inputs.probes(3, cfg.nA, cfg.l)])
    th = w.wc4d_sketch(S.ctx, w.REVD, cfg.k, m + cfg.l - cfg.k, 1, 0,
                       torch.as_tensor(G, device="cuda"), w.FP64)
    p = __import__("problems").oracle_problem(cfg, xb=tw.xb)
    Uo, tho = oracle.revd(p, cfg.k, G, q=1)
    assert np.allclose(th, tho, rtol=1e-9)
    S.close()
