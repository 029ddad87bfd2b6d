"""The benchmark's multi-GPU path (one independent replica per rank, weak
scaling, barrier + max over ranks, rank 0 reports) with two gloo ranks on CPU."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    try:
        import torch.distributed as dist
        import bench
        w, r, _ = bench.dist_init(world, backend="gloo")
        t_rank = 0.5 + rank                      # per-rank device time of the timed steps
        t_max = bench.max_over_ranks(w, t_rank)
        bench.barrier(w)
        value = bench.job_throughput(w, 3, t_max)
        seed = bench.replica_seed(r)
        # the reference arm: rank 0 alone runs and prints; others exit quietly
        out = io.StringIO()
        os.environ["WORLD_SIZE"], os.environ["RANK"] = str(world), str(rank)
        if r != 0:
            with redirect_stdout(out):
                bench.run_reference(None, None)
        dist.destroy_process_group()
        q.put((r, w, t_max, value, seed, out.getvalue()))
    except Exception as e:   # reported to the parent
        q.put(("error", repr(e)))


def test_two_replicas_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(r[0] != "error" for r in res), res
    res.sort()
    for rank, w, t_max, value, seed, out in res:
        assert w == world
        assert t_max == pytest.approx(1.5)          # the slowest replica's time, on every rank
        assert value == pytest.approx(2 * 3 / 1.5)  # whole-job inner loops per second
        assert seed == rank                          # independent problems
        assert out == ""                             # only rank 0 prints
    assert len({r[4] for r in res}) == world


def test_single_process_defaults(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1) == (1, 0, 0)
    assert bench.max_over_ranks(1, 2.5) == 2.5
    assert bench.job_throughput(1, 4, 2.0) == 2.0
