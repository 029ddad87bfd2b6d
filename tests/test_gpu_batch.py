"""Batched inner loops (independent uneven windows on their own streams,
driven concurrently): identical to running the same instances one at a
time, and each solution matches the FP64 oracle's."""
import numpy as np
import pytest

import oracle
from paper_2101_07249_gb300 import inputs
from problems import oracle_problem

torch = pytest.importorskip("torch")
w = pytest.importorskip("paper_2101_07249_gb300")
pytestmark = pytest.mark.gpu


def host(t):
    return t.double().cpu().numpy()


def test_batch_is_serial_and_matches_oracle():
    cfgs = inputs.batch_configs(seed=3, count=5, sizes=(128, 256), N_range=(3, 6), K_range=(16, 40))
    streams = [torch.cuda.Stream() for _ in cfgs]
    twins = [inputs.twin(c) for c in cfgs]
    solvers = [w.Solver(c, tw, M_shared=True, stream=s.cuda_stream) for c, tw, s in zip(cfgs, twins, streams)]
    xs = [torch.zeros(c.nA, dtype=torch.float64, device="cuda") for c in cfgs]
    ctxs = [S.ctx for S in solvers]
    ks, ls = [c.k for c in cfgs], [c.l for c in cfgs]
    seeds = [100 + i for i in range(len(cfgs))]
    torch.cuda.synchronize()
    it_c, rr_c, st_c = w.wc4d_batch_inner_loop(ctxs, w.REVD, ks, ls, 1, seeds, 1e-9, 5000, w.MIXED, xs, workers=5)
    x_c = [host(x) for x in xs]
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    it_s, rr_s, st_s = w.wc4d_batch_inner_loop(ctxs, w.REVD, ks, ls, 1, seeds, 1e-9, 5000, w.MIXED, xs, workers=1)
    assert st_c == [w.OK] * len(cfgs) and st_s == st_c
    assert it_c == it_s and rr_c == rr_s
    for a, x in zip(x_c, xs):
        assert np.array_equal(a, host(x))          # concurrency does not change any instance's arithmetic
    for c, tw, a, rr in zip(cfgs, twins, x_c, rr_c):
        assert rr <= 1e-9
        p = oracle_problem(c, xb=tw.xb)
        b = oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))
        xo = oracle.pcg(p, b, tol=1e-12, maxit=5000)["x"]
        assert np.linalg.norm(a - xo) / np.linalg.norm(xo) <= 1e-5
    for S in solvers:
        S.close()


def test_batch_rejects_shared_streams():
    cfgs = inputs.batch_configs(seed=4, count=2, sizes=(128,), N_range=(3, 3), K_range=(16, 16))
    s = torch.cuda.Stream()
    solvers = [w.Solver(c, inputs.twin(c), M_shared=True, stream=s.cuda_stream) for c in cfgs]
    xs = [torch.zeros(c.nA, dtype=torch.float64, device="cuda") for c in cfgs]
    with pytest.raises(w.WC4DError):
        w.wc4d_batch_inner_loop([S.ctx for S in solvers], w.REVD, [8, 8], [8, 8], 1, [1, 2], 1e-6, 100, w.MIXED, xs)
    for S in solvers:
        S.close()


def test_library_streams_for_many_instances():
    """More instances than torch's stream pool holds (32): library-created
    streams are distinct; a shared stream is rejected with a message."""
    cfgs = inputs.batch_configs(seed=5, count=36, sizes=(64,), N_range=(2, 3), K_range=(12, 16))
    streams = [w.wc4d_stream_create() for _ in cfgs]
    assert len(set(streams)) == len(streams)
    solvers = [w.Solver(c, inputs.twin(c), M_shared=True, stream=s) for c, s in zip(cfgs, streams)]
    xs = [torch.zeros(c.nA, dtype=torch.float64, device="cuda") for c in cfgs]
    ctxs = [S.ctx for S in solvers]
    torch.cuda.synchronize()
    it, rr, st = w.wc4d_batch_inner_loop(ctxs, w.REVD, [c.k for c in cfgs], [c.l for c in cfgs], 1,
                                         list(range(len(cfgs))), 1e-8, 5000, w.MIXED, xs, workers=8)
    assert all(r <= 1e-8 for r in rr)
    shared = w.Solver(cfgs[0], inputs.twin(cfgs[0]), M_shared=True, stream=streams[0])
    with pytest.raises(w.WC4DError, match="shares its stream"):
        w.wc4d_batch_inner_loop([ctxs[0], shared.ctx], w.REVD, [cfgs[0].k, cfgs[0].k], [cfgs[0].l, cfgs[0].l], 1,
                                [0, 1], 1e-8, 100, w.MIXED, [xs[0], xs[1]], workers=2)
    shared.close()
    for S in solvers:
        S.close()
    for s in streams:
        w.wc4d_stream_destroy(s)
