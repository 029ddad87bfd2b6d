"""Seeded synthetic inputs shared by the library's callers, the tests and the
benchmark.

This module holds the problem configurations (sizes and physical constants)
and seeded random draws.  It contains none of the method's arithmetic: no
propagator, covariance square root, Hessian product, eigensolver,
preconditioner or CG step.  The CUDA library and the CPU oracle each build
those from these inputs with their own code.

Synthetic twin recipe (identical-twin experiment of Section 5):
  * advection-diffusion truth: the exact solution of the continuous periodic
    equation u_t + c u_z = kappa u_zz for a random smooth Fourier-series
    initial state (so the discrete Crank-Nicolson model differs slightly
    from the truth, a genuine model error);
  * Lorenz-96 truth: a high-accuracy scipy ODE integration (DOP853) of the
    Lorenz-96 equations from a spun-up state;
  * background = truth at t_0 plus a smooth random field of variance
    sigma_b^2;  observations = truth at the observed points plus white
    noise of variance sigma_o^2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SOAR, GAUSS, DIAG = 0, 1, 2
MODEL_ADVDIFF, MODEL_L96 = "advdiff", "l96"


@dataclasses.dataclass(frozen=True)
class Config:
    """One inner-loop problem (Section 2) plus the sketch/CG settings."""
    name: str
    model: str
    n: int
    N: int
    steps: int
    dt: float
    kappa: float = 0.0
    u: float = 0.0
    F: float = 8.0
    b_kind: int = SOAR
    b_var: float = 1.0
    b_L: float = 5.0          # correlation length in grid points
    q_kind: int = SOAR
    q_var: float = 0.1
    q_L: float = 5.0
    obs_stride: int = 5
    obs_t0: int = 1
    sigma_o2: float = 0.01
    k: int = 10
    l: int = 5
    q_power: int = 1
    tol: float = 1e-6
    maxit: int = 5000
    seed: int = 0

    @property
    def nA(self) -> int:
        return self.n * (self.N + 1)

    @property
    def K(self) -> int:
        return self.k + self.l

    @property
    def obs_per_time(self) -> int:
        return (self.n + self.obs_stride - 1) // self.obs_stride

    @property
    def nobs(self) -> int:
        return max(self.N + 1 - self.obs_t0, 0) * self.obs_per_time

    def replace(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


# Plain FP64 tiny window: n=100 on [0,1), N=5 subwindows of 10 Crank-Nicolson
# steps, SOAR(L=0.05) covariances, every 5th point observed, REVD k=10 l=5 q=1.
TINY = Config(name="advdiff_n100_N5", model=MODEL_ADVDIFF, n=100, N=5, steps=10, dt=0.01,
              kappa=1e-3, u=0.5, b_kind=SOAR, b_var=1.0, b_L=0.05 * 100,
              q_kind=SOAR, q_var=0.1, q_L=0.05 * 100, obs_stride=5, obs_t0=1,
              sigma_o2=0.01, k=10, l=5, q_power=1)

# Large linear window: n=4096, N=40 (control dimension 167936), SOAR(L=0.02),
# every 8th point observed, 256 Gaussian probes (k=240, l=16).
LARGE = Config(name="advdiff_n4096_N40", model=MODEL_ADVDIFF, n=4096, N=40, steps=10, dt=0.01,
               kappa=1e-3, u=0.5, b_kind=SOAR, b_var=1.0, b_L=0.02 * 4096,
               q_kind=SOAR, q_var=0.1, q_L=0.02 * 4096, obs_stride=8, obs_t0=1,
               sigma_o2=0.01, k=240, l=16, q_power=1)

# The same window shortened to N=8 subwindows (control dimension 36864): a
# profiling case that keeps the device footprint to a few GB.
MEDIUM = LARGE.replace(name="advdiff_n4096_N8", N=8)

# Nonlinear Lorenz-96: n=8192, F=8, RK4 dt=0.025, 8 steps per subwindow, N=40,
# B = 0.5 Gaussian(L=4 points), Q = 0.05 I, every 4th variable observed, R = 0.1 I.
L96 = Config(name="l96_n8192_N40", model=MODEL_L96, n=8192, N=40, steps=8, dt=0.025, F=8.0,
             b_kind=GAUSS, b_var=0.5, b_L=4.0, q_kind=DIAG, q_var=0.05, q_L=1.0,
             obs_stride=4, obs_t0=1, sigma_o2=0.1, k=240, l=16, q_power=1)

CONFIGS = {c.name: c for c in (TINY, MEDIUM, LARGE, L96)}


def batch_configs(seed: int = 0, count: int = 64, sizes=(256, 512, 1024, 2048, 4096),
                  N_range=(10, 80), K_range=(32, 256), l: int = 8):
    """Uneven advection-diffusion windows (the physics of LARGE, correlation
    lengths kept in domain units): n uniform over `sizes`, N uniform in
    N_range, sketch width K = k + l uniform in K_range, instance i seeded
    with i (its truth, background, observations and probes)."""
    g = np.random.default_rng([int(seed), 4])
    out = []
    for i in range(count):
        n = int(g.choice(sizes))
        N = int(g.integers(N_range[0], N_range[1] + 1))
        K = int(g.integers(K_range[0], K_range[1] + 1))
        cfg = scaled(LARGE, n, N, K - l, l).replace(name=f"batch{i}_n{n}_N{N}_K{K}", seed=i)
        out.append(cfg)
    return out


def scaled(cfg: Config, n: int, N: int, k: int, l: int, **kw) -> Config:
    """The same physics on a smaller grid/window, correlation lengths kept in
    domain units (advection-diffusion) or grid points (Lorenz-96)."""
    if cfg.model == MODEL_ADVDIFF:
        kw.setdefault("b_L", cfg.b_L * n / cfg.n)
        kw.setdefault("q_L", cfg.q_L * n / cfg.n)
    return cfg.replace(name=f"{cfg.name}_scaled_n{n}_N{N}", n=n, N=N, k=k, l=l, **kw)


# --------------------------------------------------------------------------
# Seeded draws
# --------------------------------------------------------------------------
def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def probes(seed: int, nA: int, K: int) -> np.ndarray:
    """An explicit Gaussian probe block (K, nA) from numpy's generator; used when
    a test passes the same probes to both implementations."""
    return rng(seed, 7).standard_normal((K, nA))


def block(seed: int, nA: int, K: int, stream: int = 11) -> np.ndarray:
    """A generic random block (K, nA) for operator tests."""
    return rng(seed, stream).standard_normal((K, nA))


def _smooth_field(g: np.random.Generator, n: int, L: float, var: float) -> np.ndarray:
    """Periodic random field with a Gaussian spectral envelope of width ~1/L,
    scaled to the requested pointwise variance."""
    k = np.fft.rfftfreq(n) * n                      # wavenumbers 0..n/2
    env = np.exp(-0.25 * (2.0 * math.pi * k * L / n) ** 2)
    coef = (g.standard_normal(len(k)) + 1j * g.standard_normal(len(k))) * env
    coef[0] = 0.0
    f = np.fft.irfft(coef, n)
    s = f.std()
    return f * (math.sqrt(var) / s if s > 0 else 0.0)


def _advdiff_truth(cfg: Config, g: np.random.Generator, times: np.ndarray) -> np.ndarray:
    """Exact solution of u_t + c u_z = kappa u_zz on [0,1) for a random
    Fourier-series initial state (modes 1..16, smooth envelope); rows = times."""
    m = np.arange(1, 17)
    amp = 2.0 * g.standard_normal(len(m)) * np.exp(-0.5 * (m / 4.0) ** 2)
    phase = g.uniform(0.0, 2.0 * math.pi, len(m))
    z = np.arange(cfg.n) / cfg.n
    out = np.zeros((len(times), cfg.n))
    for i, t in enumerate(times):
        decay = np.exp(-cfg.kappa * (2.0 * math.pi * m) ** 2 * t)
        arg = 2.0 * math.pi * np.outer(m, z - cfg.u * t) + phase[:, None]
        out[i] = (amp * decay) @ np.cos(arg)
    return out


def _l96_rhs(F):
    def f(_t, x):
        return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F
    return f


def _l96_truth(cfg: Config, g: np.random.Generator, times: np.ndarray, spinup: float) -> np.ndarray:
    from scipy.integrate import solve_ivp
    x0 = cfg.F + 0.01 * g.standard_normal(cfg.n)
    f = _l96_rhs(cfg.F)
    sp = solve_ivp(f, (0.0, spinup), x0, method="DOP853", rtol=1e-9, atol=1e-9)
    xs = sp.y[:, -1]
    tr = solve_ivp(f, (0.0, float(times[-1])), xs, method="DOP853", rtol=1e-10, atol=1e-10,
                   t_eval=times)
    return tr.y.T.copy()


@dataclasses.dataclass
class Twin:
    """Identical-twin inputs: background x^b (n), observations y (nobs, time-major
    over t = obs_t0..N, points s = 0, stride, ...), and the truth at t_0..t_N."""
    xb: np.ndarray
    y: np.ndarray
    truth: np.ndarray


def twin(cfg: Config, spinup: float = 50.0) -> Twin:
    g = rng(cfg.seed, 1)
    times = np.arange(cfg.N + 1) * cfg.steps * cfg.dt
    if cfg.model == MODEL_ADVDIFF:
        truth = _advdiff_truth(cfg, g, times)
        bg_L = cfg.b_L
    else:
        truth = _l96_truth(cfg, g, times, spinup)
        bg_L = cfg.b_L
    xb = truth[0] + _smooth_field(g, cfg.n, bg_L, cfg.b_var)
    per = cfg.obs_per_time
    y = np.zeros(cfg.nobs)
    k = 0
    for t in range(cfg.obs_t0, cfg.N + 1):
        pts = truth[t, ::cfg.obs_stride][:per]
        y[k:k + per] = pts + math.sqrt(cfg.sigma_o2) * g.standard_normal(per)
        k += per
    return Twin(xb=xb, y=y, truth=truth)
