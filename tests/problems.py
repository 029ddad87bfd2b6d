"""Oracle problem builders for the tests (oracle side only)."""
import numpy as np

import oracle
from paper_2101_07249_gb300 import inputs


def cov_sqrt_rows(cfg):
    bs, _, _ = oracle.cov_sqrt_row(cfg.b_kind, cfg.n, cfg.b_L, cfg.b_var)
    qs, _, _ = oracle.cov_sqrt_row(cfg.q_kind, cfg.n, cfg.q_L, cfg.q_var)
    return bs, qs


def oracle_problem(cfg, mode="stepping", xb=None, spinup_traj=None):
    """The oracle's Problem for a config.  mode: 'stepping' (Crank-Nicolson
    solves), 'dense' (propagator built by stepping unit vectors) or, for
    Lorenz-96, the TLM along the RK4 trajectory from xb."""
    bs, qs = cov_sqrt_rows(cfg)
    common = dict(n=cfg.n, N=cfg.N, Bsqrt=bs, Qsqrt=qs, sigma_o2=cfg.sigma_o2,
                  obs_stride=cfg.obs_stride, obs_t0=cfg.obs_t0, steps=cfg.steps, dt=cfg.dt)
    if cfg.model == inputs.MODEL_ADVDIFF:
        if mode == "dense":
            M = oracle.advdiff_dense(cfg.n, cfg.kappa, cfg.u, cfg.dt, cfg.steps)
            return oracle.Problem(model=oracle.MODEL_DENSE, M=M, M_shared=True, **common)
        return oracle.Problem(model=oracle.MODEL_ADVDIFF, kappa=cfg.kappa, u=cfg.u, **common)
    assert xb is not None
    traj = oracle.l96_run(xb, cfg.F, cfg.dt, cfg.N * cfg.steps)
    return oracle.Problem(model=oracle.MODEL_L96, F=cfg.F, traj=traj, **common)


def dense_A(p):
    """A built column by column with the oracle's Hessian product."""
    return oracle.hvp(p, np.eye(p.nA)).T.copy()
