#!/usr/bin/env python
"""Benchmark of the randomised-LMP inner loop of weak-constraint 4D-Var.

One step = one inner loop (Section 4): Gaussian probes, REVD with one power
iteration (3 block Hessian products of 256 columns), CholeskyQR2, Rayleigh-
Ritz, spectral LMP, PCG to relative residual 1e-6, on the large linear window
(periodic advection-diffusion, n = 4096, N = 40 subwindows, control dimension
167936, a dense propagator per subwindow).  The chosen form is the mixed
path (FP32 sweeps and CG, FP64 Gram/Cholesky/Jacobi/CG scalars and true-
residual refinement); the plain FP64 path is timed beside it.

Prints ONE JSON line (rank 0).  value = inner loops per second over all ranks
(one independent replica per GPU, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inner-loop time to rel-res 1e-6 and Hessian-vec products/s, mixed vs FP64 plain"

# DRAM bytes per launch of the dominant kernel from `ncu` (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel class and workload; see profiles/.
# k_gemv_sweep_staged<2>: measured on the N = 8 window (8 subwindow GEMVs) and
# scaled by 40/8 to the N = 40 window (traffic grows with the number of
# subwindows).  None whenever the kernel has changed since the counters were
# taken.
NCU_TRAFFIC = {("gemv_sweep_f32", "advdiff_n4096_N40"): 540.49e6 * 40 / 8}

# Column Hessian products one mixed inner loop issues on the large window:
# REVD with one power iteration (3 block products of k + l = 256 columns),
# ~111 PCG iterations and 2 FP64 true residuals.  Used only to express the
# CPU oracle's column-product rate in inner loops per second.
INNER_LOOP_COLUMN_PRODUCTS = 3 * 256 + 111 + 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), float(pk["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- distributed
def dist_init(n_gpus, backend=None):
    """One process per GPU (torchrun env); NCCL on GPUs, gloo when asked (CPU tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = backend or "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    """Largest v over the ranks (the job's time is its slowest replica's)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Each replica solves its own independent problem (weak scaling)."""
    return rank


def job_throughput(world, steps, t_max):
    """Inner loops per second of the whole job: every rank ran `steps`."""
    return world * steps / t_max


def hvp_block_roofline(cfg, t_s):
    """The K-column block Hessian product against both roofs: the propagator
    GEMMs of both sweeps (2 N x 2 n^2 K flop) against the TF32 tensor peak
    (the measured BF16 burst x the nominal TF32/BF16 ratio 1.1/2.25), and the
    TF32-rounded FP32 propagators read once per sweep plus the block read and
    written (2 N n^2 x 4 + 2 nA K x 4 bytes) against the measured HBM copy."""
    hbm, bf16, _, src = _peaks()
    flops = 2.0 * cfg.N * 2.0 * cfg.n * cfg.n * cfg.K
    nbytes = 2.0 * cfg.N * cfg.n * cfg.n * 4 + 2.0 * cfg.nA * cfg.K * 4
    tf32 = bf16 * 1.1 / 2.25
    return {"tflops": flops / t_s / 1e12, "tf32_peak": tf32, "tensor_frac": flops / t_s / 1e12 / tf32,
            "gbs": nbytes / t_s / 1e9, "hbm_peak": hbm, "hbm_frac": nbytes / t_s / 1e9 / hbm, "peak_source": src}


def workload_config(cfg, method):
    """The workload both arms report (the same dict in both lines)."""
    return {"workload": cfg.name, "n": cfg.n, "N": cfg.N, "nA": cfg.nA, "K": cfg.K, "k": cfg.k, "l": cfg.l,
            "method": method, "q_power": cfg.q_power, "tol": cfg.tol,
            "propagators": "one dense matrix per subwindow",
            "l2": (f"inputs larger than L2 (propagators {cfg.N * cfg.n * cfg.n * 4 / 1e9:.2f} GB FP32, "
                   f"{cfg.N * cfg.n * cfg.n * 8 / 1e9:.2f} GB FP64)"),
            "parallelism": "replicas"}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_column_rate(cfg, cols=16):
    """Column Hessian products per second of the FP64 oracle (plain C, OpenMP
    over columns) on a `cols`-column block of the large window, dense-
    propagator mode (the same algorithm as the library's sweeps)."""
    import oracle
    from paper_2101_07249_gb300 import inputs
    M = oracle.advdiff_dense(cfg.n, cfg.kappa, cfg.u, cfg.dt, cfg.steps)
    p = oracle.Problem(cfg.n, cfg.N, oracle.MODEL_DENSE, oracle.cov_sqrt_row(cfg.b_kind, cfg.n, cfg.b_L, cfg.b_var)[0],
                       oracle.cov_sqrt_row(cfg.q_kind, cfg.n, cfg.q_L, cfg.q_var)[0], cfg.sigma_o2, cfg.obs_stride, cfg.obs_t0,
                       M=M, M_shared=True)
    X = inputs.block(1, cfg.nA, cols)
    t0 = time.perf_counter()
    oracle.hvp(p, X)
    dt = time.perf_counter() - t0
    return cols / dt, dt


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def oracle_tiny_inner_loop(threads):
    """One full inner loop of the FP64 oracle on the tiny window (n = 100, N =
    5: REVD q = 1 with 15 Philox probes, spectral LMP, PCG to 1e-6) with
    `threads` OpenMP threads; returns (seconds, PCG iterations)."""
    import oracle
    from paper_2101_07249_gb300 import inputs
    cfg = inputs.TINY
    tw = inputs.twin(cfg)
    M = oracle.advdiff_dense(cfg.n, cfg.kappa, cfg.u, cfg.dt, cfg.steps)
    p = oracle.Problem(cfg.n, cfg.N, oracle.MODEL_DENSE, oracle.cov_sqrt_row(cfg.b_kind, cfg.n, cfg.b_L, cfg.b_var)[0],
                       oracle.cov_sqrt_row(cfg.q_kind, cfg.n, cfg.q_L, cfg.q_var)[0], cfg.sigma_o2, cfg.obs_stride,
                       cfg.obs_t0, M=M, M_shared=True)
    b = oracle.rhs(p, oracle.innovation(p, tw.xb, tw.y))
    prev = oracle.threads()
    oracle.threads(threads)
    try:
        best, iters = None, 0
        for rep in range(3):
            t0 = time.perf_counter()
            G = oracle.gaussian(rep, cfg.nA, cfg.K)
            U, th = oracle.revd(p, cfg.k, G, q=cfg.q_power)
            r = oracle.pcg(p, b, U, th, tol=cfg.tol, maxit=cfg.maxit)
            dt = time.perf_counter() - t0
            best, iters = (dt, r["iters"]) if best is None or dt < best else (best, iters)
    finally:
        oracle.threads(prev)
    return best, iters


def oracle_timings(cfg, sample_cols, sample_s, products):
    """The FP64 oracle timed on this machine's host cores: the tiny window's
    whole inner loop on one thread and on all cores, and the large window's
    block Hessian product and inner loop, extrapolated from a measured
    `sample_cols`-column product (the full ones take minutes)."""
    import oracle
    allc = oracle.threads()
    t1, it1 = oracle_tiny_inner_loop(1)
    ta, ita = oracle_tiny_inner_loop(allc)
    per_col = sample_s / sample_cols
    return {"cores": allc,
            "tiny_inner_loop": {"workload": "advdiff_n100_N5", "threads_1_s": t1, f"threads_{allc}_s": ta,
                                "pcg_iters": ita, "measured": True},
            "large_block_hvp": {"workload": cfg.name, "K": cfg.K, "s": per_col * cfg.K, "measured_columns": sample_cols,
                                "measured_s": sample_s, "extrapolated_from": f"{sample_cols} columns"},
            "large_inner_loop": {"workload": cfg.name, "s": per_col * products, "column_products": products,
                                 "extrapolated_from": f"{sample_cols}-column product; sketch linear algebra not counted"}}


def run_reference(args, cfg):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    One step = one measured sample of the workload: a block Hessian product
    of 8 columns of the large window (dense-propagator mode).  ms_per_step is
    that sample's measured time; value converts the measured column rate to
    inner loops per second by the column products one inner loop issues."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cols = 8
    products = INNER_LOOP_COLUMN_PRODUCTS if cfg.name == "advdiff_n4096_N40" else 3 * cfg.K + 100
    times = []
    for i in range(args.warmup + args.steps):
        rate, dt = oracle_column_rate(cfg, cols=cols)
        if i >= args.warmup:
            times.append(dt)
    col_rate = cols * len(times) / sum(times)
    value = col_rate / products
    sample = (f"each step: one {cols}-column block Hessian product of the {cfg.name} window (FP64 oracle, dense "
              f"propagator mode), {1e3 * statistics.mean(times):.0f} ms measured; value = measured column rate / "
              f"{products} column products per inner loop (sketch linear algebra not counted)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "inner_loops/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "ms_per_step_is": f"the measured {cols}-column sample",
            "inner_loop_s_extrapolated": 1.0 / value if value else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(cfg, args.method), "precision": "fp64",
            "cpu_baseline": {"value": value, "unit": "inner_loops/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "inner_loops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- Lorenz-96 window
def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak from the unit counts and the clock: 152 SMs x 128 lanes x 2 flop per cycle."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def lorenz96_window(w, inputs, rank, stream, outer_loops=3, maxit=100, sm_mhz=2070.0):
    """The nonlinear window (n = 8192, N = 40 subwindows of 8 RK4 steps,
    K = 256): three outer loops, each a mixed inner loop (REVD q = 1, LMP,
    PCG) followed by the outer update (eq. 3), plus the block Hessian
    product rate.  As in the paper's Lorenz-96 experiments (Section 5.2)
    PCG stops after 100 iterations or at relative residual 1e-6: this window
    spans 8 model time units, its Hessian's largest eigenvalues are ~1e17
    and 1e-6 is out of reach of any CG; the relative residual and the
    quadratic-cost decrease reached are reported.  The sweeps are RK4
    tangent-linear / adjoint stencils: FP32 ALU work, reported against the
    FP32 FMA peak from the unit counts and the sampled SM clock."""
    import torch
    c3 = inputs.L96.replace(seed=replica_seed(rank))
    tw3 = inputs.twin(c3)
    S3 = w.Solver(c3, tw3)
    x3 = torch.zeros(c3.nA, dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loops = []
    for j in range(outer_loops):
        torch.cuda.synchronize()
        e0.record(stream)
        th = w.wc4d_sketch(S3.ctx, w.REVD, c3.k, c3.l, c3.q_power, 10 + j, None, w.MIXED)
        it, rr, qcf, st = w.wc4d_pcg(S3.ctx, x3, c3.tol, maxit, 1, 0, w.MIXED, qcf=True, raise_on_noconv=False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_inner = e0.elapsed_time(e1)
        e0.record(stream)
        w.wc4d_outer_update(S3.ctx, x3)
        e1.record(stream)
        torch.cuda.synchronize()
        loops.append({"inner_loop_ms": t_inner, "pcg_iters": it, "relres": rr,
                      "qcf_decrease": float(sum(qcf)) if qcf is not None else None,
                      "theta_max": float(th[0]), "theta_k": float(th[-1]), "outer_update_ms": e0.elapsed_time(e1)})
    K = c3.K
    Xb = torch.randn(K, c3.nA, dtype=torch.float32, device="cuda")
    Yb = torch.empty_like(Xb)
    w.wc4d_hvp(S3.ctx, Xb, Yb, K, c3.nA, w.MIXED)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        w.wc4d_hvp(S3.ctx, Xb, Yb, K, c3.nA, w.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    t_hvp = e0.elapsed_time(e1) / 3e3
    # flop model per column: 2 sweeps x N x steps RK4 steps x n variables x
    # (4 stages x (6-flop tangent stencil + 2-flop stage update) + 8-flop combination)
    flop_col = 2.0 * c3.N * c3.steps * c3.n * (4 * 8 + 8)
    S3.close()
    return {"workload": c3.name, "nA": c3.nA, "K": K, "pcg_maxit": maxit, "outer_loops": loops,
            "hvp_block_ms": 1e3 * t_hvp, "hvp_columns_per_s": K / t_hvp,
            "hvp_alu": {"bound": "alu", "achieved_tflops": flop_col * K / t_hvp / 1e12,
                        "peak_tflops": fp32_peak_tflops(sm_mhz),
                        "frac": flop_col * K / t_hvp / 1e12 / fp32_peak_tflops(sm_mhz),
                        "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (median SM clock of "
                                       "the timed region)"}}


def profile_l96_hvp(inputs, K=256, blocks=2):
    """A short program for ncu captures of the Lorenz-96 stencil sweeps: the
    n = 8192 window cut to N = 2 subwindows, two K-column FP32 Hessian blocks
    (K = 256: the sketch's block, two columns per CTA; K = 1: the PCG
    matvec, one CTA)."""
    import torch
    import paper_2101_07249_gb300 as w
    w.load()
    c = inputs.L96.replace(N=2, name="l96_n8192_N2")
    S = w.Solver(c, inputs.twin(c, spinup=2.0))
    gen = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(K, c.nA, dtype=torch.float32, device="cuda", generator=gen)
    Y = torch.empty_like(X)
    w.wc4d_launch_count(reset=True)
    for _ in range(blocks):
        w.wc4d_hvp(S.ctx, X, Y, K, c.nA, w.MIXED)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": c.name, "K": K, "blocks": blocks, "gpu_launches": w.wc4d_launch_count()}))
    S.close()


# ---------------------------------------------------------------- learned sketch
LEARNED_WEIGHTS = os.path.join(ROOT, "paper_2101_07249_gb300", "learned", "l96_n8192_N10_m64.npz")


def learned_windows(w, inputs, stream, seeds=(30000, 30001, 30002, 30003), m=64, l=32, maxit=5000):
    """Lorenz-96 windows (n = 8192, N = 10, held-out seeds): the Gaussian
    sketch (REVD q = 1, m + l probes) against the learned proposal (m network
    columns + l Gaussian columns through the same REVD), each followed by
    mixed PCG to 1e-6.  Gate (paper_2101_07249_gb300.learned.accept): the
    learned block is used when the sum of its top-m Ritz values is at least
    that of the Gaussian block of the same width, else the Gaussian sketch is.
    Each window reports both blocks' PCG iterations (the learned one is run
    whatever the gate decides, to check the decision) and the gated path's.
    Four held-out seeds."""
    import torch
    from paper_2101_07249_gb300.learned import accept as gate
    if not os.path.exists(LEARNED_WEIGHTS):
        return None
    z = np.load(LEARNED_WEIGHTS)
    wdev = torch.as_tensor(np.concatenate([z[f"W{i}"].ravel() for i in range(4)]).view(np.int16), device="cuda")
    bdev = torch.as_tensor(np.concatenate([z[f"b{i}"] for i in range(4)]).astype(np.float32), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    rows = []
    for sd in seeds:
        cfg = inputs.L96.replace(N=10, name=f"l96_n8192_N10_s{sd}", seed=sd, k=m, l=l)
        tw = inputs.twin(cfg, spinup=5.0)
        S = w.Solver(cfg, tw)
        x = torch.zeros(cfg.nA, dtype=torch.float64, device="cuda")
        th_g, t_sk_g = timed(lambda: w.wc4d_sketch(S.ctx, w.REVD, m, l, 1, sd, None, w.MIXED))
        (it_g, rr_g, _, _), t_pcg_g = timed(lambda: w.wc4d_pcg(S.ctx, x, 1e-6, maxit, 1, 0, w.MIXED,
                                                                 raise_on_noconv=False))
        G = torch.zeros(m + l, cfg.nA, dtype=torch.float64, device="cuda")

        def learned_sketch():
            w.wc4d_learned_probes(S.ctx, wdev, bdev, m, G, cfg.nA)
            w.wc4d_gaussian(S.ctx, sd, cfg.nA, l, cfg.nA, G[m:])
            return w.wc4d_sketch(S.ctx, w.REVD, m, l, 1, sd, G, w.MIXED)

        th_l, t_sk_l = timed(learned_sketch)
        accept = gate(th_l, th_g)
        row = {"seed": sd, "gaussian": {"sketch_ms": t_sk_g, "pcg_ms": t_pcg_g, "pcg_iters": it_g, "relres": rr_g,
                                        "theta_topm_sum": float(np.sum(th_g))},
               "learned": {"sketch_ms": t_sk_l, "theta_topm_sum": float(np.sum(th_l)), "accepted": accept}}
        # the learned block's own PCG, run whether or not the gate accepts it,
        # to check the gate's decision against the CG iteration count
        x.zero_()
        (it_l, rr_l, _, _), t_pcg_l = timed(lambda: w.wc4d_pcg(S.ctx, x, 1e-6, maxit, 1, 0, w.MIXED,
                                                                 raise_on_noconv=False))
        row["learned"].update({"pcg_ms": t_pcg_l, "pcg_iters": it_l, "relres": rr_l})
        row["gated"] = {"path": "learned" if accept else "gaussian", "pcg_iters": it_l if accept else it_g,
                        "sketch_plus_pcg_ms": (t_sk_g + t_sk_l + t_pcg_l) if accept else (t_sk_g + t_sk_l + t_pcg_g)}
        rows.append(row)
        S.close()
    return {"workload": "l96_n8192_N10 (held-out seeds)", "m": m, "l": l,
            "held_out_captured": float(z["held_out_captured"]), "gaussian_captured": float(z["gaussian_captured"]),
            "windows": rows}


# ---------------------------------------------------------------- batched windows
def batched_windows(w, inputs, count, workers=16):
    """Uneven advection-diffusion windows (n in {256..4096}, N in [10, 80],
    K in [32, 256], one propagator per window): all inner loops of the batch
    (mixed path, REVD q = 1, tol 1e-6) driven concurrently, each window on
    its own stream, against the same mixed inner loops run one window after
    another (the gain of batching alone) and against looping the plain FP64
    single-window solver over the same windows.  Wall-clock times around the
    host calls."""
    import torch
    cfgs = inputs.batch_configs(seed=0, count=count)
    streams = [w.wc4d_stream_create() for _ in cfgs]   # torch's pool repeats streams past 32
    solvers = [w.Solver(c, inputs.twin(c), M_shared=True, stream=st) for c, st in zip(cfgs, streams)]
    xs = [torch.zeros(c.nA, dtype=torch.float64, device="cuda") for c in cfgs]
    ctxs = [S.ctx for S in solvers]
    ks, ls = [c.k for c in cfgs], [c.l for c in cfgs]
    torch.cuda.synchronize()
    w.wc4d_batch_inner_loop(ctxs, w.REVD, ks, ls, 1, list(range(count)), 1e-6, 5000, w.MIXED, xs, workers)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_b, rr_b, st_b = w.wc4d_batch_inner_loop(ctxs, w.REVD, ks, ls, 1, list(range(count)), 1e-6, 5000, w.MIXED, xs,
                                                workers)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    def looped(precision):
        its = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, (S, c, x) in enumerate(zip(solvers, cfgs, xs)):
            it, _ = w.wc4d_inner_loop(S.ctx, w.REVD, c.k, c.l, 1, i, 1e-6, 5000, precision, x)
            its.append(it)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, its

    t_mixed, it_m = looped(w.MIXED)      # the same mixed inner loops one window after another
    t_fp64, it_f = looped(w.FP64)
    for S in solvers:
        S.close()
    for st in streams:
        w.wc4d_stream_destroy(st)
    return {"windows": count, "workers": workers, "total_nA": int(sum(c.nA for c in cfgs)),
            "batched_mixed_s": t_batch, "looped_mixed_s": t_mixed, "looped_fp64_s": t_fp64,
            "speedup_batching": t_mixed / t_batch, "speedup_vs_looped_fp64": t_fp64 / t_batch,
            "max_relres": max(rr_b), "pcg_iters_batched": it_b, "pcg_iters_looped_mixed": it_m,
            "pcg_iters_fp64": it_f}


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wc4d", choices=["wc4d", "reference"])
    ap.add_argument("--method", default="revd", choices=["revd", "nystrom", "ritzit", "nystrom1"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the method comparison, the Lorenz-96 window and the batched windows")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="uneven windows in the batched comparison")
    ap.add_argument("--workload", default="large", choices=["large", "medium", "tiny", "l96_hvp"],
                    help="large: n=4096 N=40 (the benchmark); medium: N=8 (profiling captures); tiny: n=100 N=5; "
                         "l96_hvp: two K=256 FP32 Hessian blocks on a 2-subwindow Lorenz-96 window "
                         "(profiling captures of the stencil sweeps, with --profile-run)")
    ap.add_argument("--l96-k", type=int, default=256,
                    help="with --workload l96_hvp: columns of each Hessian block (256: the sketch's block; 1: the "
                         "PCG matvec)")
    ap.add_argument("--profile-run", action="store_true",
                    help="only --warmup inner loops and one more, then exit (a short program for ncu captures)")
    ap.add_argument("--eager", action="store_true",
                    help="with --profile-run: CG iterations as eager launches, not CUDA graphs (the same kernels; "
                         "ncu does not list the kernels inside the graphs' conditional loop)")
    args = ap.parse_args()

    from paper_2101_07249_gb300 import inputs
    if args.workload == "l96_hvp":
        if not args.profile_run:
            ap.error("--workload l96_hvp is a profiling case: give --profile-run")
        profile_l96_hvp(inputs, K=args.l96_k)
        return
    cfg = {"large": inputs.LARGE, "medium": inputs.MEDIUM, "tiny": inputs.TINY}[args.workload]
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    import paper_2101_07249_gb300 as w

    world, rank, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    w.load()
    meth = w.METHODS[args.method]
    cfg = cfg.replace(seed=replica_seed(rank))
    tw = inputs.twin(cfg)
    S = w.Solver(cfg, tw, M_shared=False)
    ctx = S.ctx
    nA = cfg.nA
    if args.profile_run and args.eager:
        w.wc4d_set_graphs(ctx, 0)
    x = torch.zeros(nA, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def inner(precision, seed):
        return w.wc4d_inner_loop(ctx, meth, cfg.k, cfg.l, cfg.q_power, seed, cfg.tol, cfg.maxit, precision, x)

    # ---- warm-up (mixed path)
    for i in range(args.warmup):
        inner(w.MIXED, 1000 + i)
    torch.cuda.synchronize()
    if args.profile_run:
        w.wc4d_launch_count(reset=True)
        it, rr = inner(w.MIXED, 0)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": cfg.name, "pcg_iters": it, "relres": rr,
                          "gpu_launches": w.wc4d_launch_count()}))
        S.close()
        return

    # ---- timed region: device-resident inputs
    clocks = ClockSampler(local)
    clocks.start()
    w.wc4d_launch_count(reset=True)
    w.wc4d_hvp_count(ctx, reset=True)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, relres = [], []
    e0.record(stream)
    for i in range(args.steps):
        it, rr = inner(w.MIXED, i)
        iters.append(it)
        relres.append(rr)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_dev = e0.elapsed_time(e1) / 1e3
    launches = w.wc4d_launch_count()
    products_block = w.wc4d_hvp_count(ctx)
    clk = clocks.stop()
    t_max = max_over_ranks(world, t_dev)
    value = job_throughput(world, args.steps, t_max)

    # ---- end to end through host buffers: H2D of x^b and y (pinned), the
    # outer-loop set-up (innovations, rhs), the inner loop, D2H of x
    xb_h = torch.from_numpy(tw.xb.copy()).pin_memory()
    y_h = torch.from_numpy(tw.y.copy()).pin_memory()
    x_h = torch.empty(nA, dtype=torch.float64).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        w.wc4d_set_background_obs(ctx, xb_h.numpy(), y_h.numpy())
        inner(w.MIXED, 100 + i)
        x_h.copy_(x)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(world, time.perf_counter() - t0)
    e2e = {"value": world * args.steps / t_e2e, "unit": "inner_loops/s",
           "h2d_bytes_per_step": 8 * (cfg.n + cfg.nobs), "d2h_bytes_per_step": 8 * nA}

    # ---- block Hessian products per second (K = 256 probe columns)
    K = cfg.K
    Xb = torch.randn(K, nA, dtype=torch.float32, device="cuda")
    Yb = torch.empty_like(Xb)
    w.wc4d_hvp(ctx, Xb, Yb, K, nA, w.MIXED)
    torch.cuda.synchronize()
    e0.record(stream)
    reps = 3
    for _ in range(reps):
        w.wc4d_hvp(ctx, Xb, Yb, K, nA, w.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    t_hvp_mixed = e0.elapsed_time(e1) / 1e3 / reps
    del Xb, Yb

    # ---- live per-kernel-class timing of one more mixed inner loop
    w.wc4d_profile(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    it_p, _ = inner(w.MIXED, 77)
    ev1.record()
    torch.cuda.synchronize()
    profiled_ms = ev0.elapsed_time(ev1)
    jacobi_sweeps = {"fp32": w.wc4d_jacobi_sweeps_fp32(ctx), "fp64": w.wc4d_jacobi_sweeps(ctx),
                     "fp32_kernel": {0: None, 1: "cluster16", 2: "cooperative"}.get(w.wc4d_jacobi_fp32_kernel(ctx))}
    classes = {}
    for ci, name in enumerate(w.PROF_CLASSES):
        ms, cnt = w.wc4d_profile_read(ctx, ci)
        if cnt:
            classes[name] = {"ms": ms, "launch_groups": cnt, "avg_us": 1e3 * ms / cnt}
    w.wc4d_profile(ctx, False)

    hbm, bf16, bf16_s, peak_src = _peaks()
    dom = max(classes, key=lambda k: classes[k]["ms"]) if classes else None
    roof = None
    n = cfg.n
    if dom == "gemv_sweep":
        # one timed group = one persistent launch of all N subwindow GEMVs
        bytes_per = cfg.N * (4 * n * n + 3 * 4 * n)           # FP32 propagators + x, C_old, C
        ach = bytes_per / (classes[dom]["avg_us"] * 1e-6) / 1e9
        tr = NCU_TRAFFIC.get(("gemv_sweep_f32", cfg.name))
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": tr, "kernel": "k_gemv_sweep_staged<2> (persistent one-column FP32 sweep, bulk-copy ring, "
                                          "N GEMVs per launch)",
                "algorithmic_bytes_per_launch": bytes_per, "peak_source": peak_src}
    elif dom in ("gemm", "tc_gemm"):
        flops = 2.0 * n * n * K
        ach = flops / (classes[dom]["avg_us"] * 1e-6) / 1e12
        if dom == "tc_gemm":
            pk = bf16 * (1.1 / 2.25)
            roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": None, "kernel": "tcgen05 TF32 sweep GEMM", "peak_source": peak_src + " x TF32/BF16"}
        else:
            sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
            pk = fp32_peak_tflops(sm_mhz)
            roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": None, "kernel": "SIMT FP32 sweep GEMM",
                    "peak_source": "152 SM x 128 FP32 lanes x 2 x median SM clock"}
    elif dom is not None:
        roof = {"bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None, "traffic": None,
                "kernel": dom}

    # ---- the plain FP64 method on the same GPU
    fp64 = None
    if not args.no_fp64:
        inner(w.FP64, 5000)
        torch.cuda.synchronize()
        e0.record(stream)
        it64, rr64 = inner(w.FP64, 5001)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        Xb = torch.randn(K, nA, dtype=torch.float64, device="cuda")
        Yb = torch.empty_like(Xb)
        e0.record(stream)
        w.wc4d_hvp(ctx, Xb, Yb, K, nA, w.FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        t_hvp64 = e0.elapsed_time(e1) / 1e3
        del Xb, Yb
        fp64 = {"inner_loop_s": t64, "pcg_iters": it64, "relres": rr64, "hvp_block_s": t_hvp64,
                "hvp_columns_per_s": K / t_hvp64}

    # ---- the three sketching methods of Section 4 and single-pass Nystrom (Section 6) on the same window
    methods, l96, batched, learned, paper_adv = None, None, None, None, None
    if not args.no_extra and args.workload == "large":
        methods = {}
        for mname in ("revd", "nystrom", "ritzit", "nystrom1"):
            # one untimed inner loop first: a method's first run grows its buffers and tunes the tile
            # shapes of products the others do not have
            w.wc4d_inner_loop(ctx, w.METHODS[mname], cfg.k, cfg.l, cfg.q_power, 554, cfg.tol, cfg.maxit, w.MIXED, x)
            torch.cuda.synchronize()
            e0.record(stream)
            it_m, rr_m = w.wc4d_inner_loop(ctx, w.METHODS[mname], cfg.k, cfg.l, cfg.q_power, 555, cfg.tol,
                                           cfg.maxit, w.MIXED, x)
            e1.record(stream)
            torch.cuda.synchronize()
            methods[mname] = {"inner_loop_ms": e0.elapsed_time(e1), "pcg_iters": it_m, "relres": rr_m,
                              "block_products": {"revd": 1 + cfg.q_power + 1, "nystrom": 2}.get(mname, 1)}
        l96 = lorenz96_window(w, inputs, rank, stream, sm_mhz=(clk or {}).get("sm_mhz") or 2070.0)
        batched = batched_windows(w, inputs, args.batch_count) if args.batch_count > 0 else None
        learned = learned_windows(w, inputs, stream)
        from paper_2101_07249_gb300 import paper_setups
        paper_adv = {"advection": paper_setups.spectral_study(), "lorenz96": paper_setups.lorenz96_study(),
                     "lorenz96_networks": paper_setups.lorenz96_networks()}

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        products = 3 * K + statistics.mean(iters) + 2
        cols = 16
        rate, dt = oracle_column_rate(cfg, cols=cols)
        timings = oracle_timings(cfg, cols, dt, products)
        cpu = {"value": rate / products, "unit": "inner_loops/s", "cores": omp_threads(), "kind": "oracle",
               "sample": (f"{cols}-column block Hessian product ({dt:.1f} s measured, FP64 oracle, dense-propagator "
                          f"mode) scaled by {products:.0f} column products per inner loop; sketch linear algebra "
                          "not counted"),
               "timings": timings}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "inner_loops/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(cfg, args.method), "precision": "mixed",
            "inner_loop_ms": 1e3 * t_max / args.steps,
            "pcg_iters": iters, "relres": relres,
            "block_products_per_step": products_block / args.steps,
            "hvp_columns_per_s": K / t_hvp_mixed, "hvp_block_ms": 1e3 * t_hvp_mixed,
            "hvp_block_roofline": hvp_block_roofline(cfg, t_hvp_mixed),
            "fp64_plain": fp64,
            "speedup_vs_fp64": (fp64["inner_loop_s"] / (t_max / args.steps)) if fp64 else None,
            "kernel_classes": classes,
            "jacobi_sweeps": jacobi_sweeps,
            "profiled_inner_loop_ms": profiled_ms,
            "unclassified_ms": profiled_ms - sum(v["ms"] for v in classes.values()),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "methods": methods,
            "lorenz96": l96,
            "batched": batched,
            "learned_sketch": learned,
            "paper_windows": paper_adv,
        }
        print(json.dumps(line))
    S.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
