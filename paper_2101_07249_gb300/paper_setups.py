"""The paper's own linear advection window (Section 5.1), built through the
C-ABI, and the spectral study the section reports (its Ritz-value and
preconditioned-spectrum figures).

Window: u_t + u_z = 0 on [0, 1), periodic, n = 40 points, first-order upwind
steps with Courant number 0.8, N = 50 subwindows of one step each, every 4th
variable observed at every 5th step (t = 5, 10, .., 50: 100 observations),
sigma_o = 0.05, B = 0.1^2 SOAR(10 dz), Q_t = 0.05^2 C_q with length 10 dz.
The paper's C_q is a "Laplacian" correlation it does not define; SOAR with the
same length scale stands in for it.  Identical twin: truth from the Gaussian
initial state 6 exp(-(z - 0.5)^2 / (2 0.1^2)), background = truth + B^{1/2}
noise, observations = truth + sigma_o noise (seeded).
"""
from __future__ import annotations

import numpy as np

N_ADV, n_ADV, COURANT = 50, 40, 0.8
SIG_O, SIG_Q, SIG_B, LEN = 0.05, 0.05, 0.1, 10.0
OBS_STRIDE, OBS_T0, OBS_TSTRIDE = 4, 5, 5


def upwind_propagator(n: int = n_ADV, courant: float = COURANT) -> np.ndarray:
    """One first-order upwind step of u_t + u_z = 0 (wind to the right,
    periodic): u_i <- (1 - C) u_i + C u_{i-1}, as a row-major n x n matrix."""
    M = (1.0 - courant) * np.eye(n)
    M[np.arange(n), (np.arange(n) - 1) % n] += courant
    return M


def soar_row(n: int, variance: float, length: float) -> np.ndarray:
    r = np.minimum(np.arange(n), n - np.arange(n)).astype(np.float64)
    return variance * (1.0 + r / length) * np.exp(-r / length)


def advection_twin(seed: int = 0):
    """Truth (N + 1, n), background x^b (n) and observations y (100,)."""
    g = np.random.default_rng([int(seed), 51])
    z = np.arange(n_ADV) / n_ADV
    M = upwind_propagator()
    truth = np.zeros((N_ADV + 1, n_ADV))
    truth[0] = 6.0 * np.exp(-(z - 0.5) ** 2 / (2 * 0.1 ** 2))
    for t in range(N_ADV):
        truth[t + 1] = M @ truth[t]
    row = soar_row(n_ADV, SIG_B ** 2, LEN)
    Bm = np.array([np.roll(row, i) for i in range(n_ADV)])
    lam, V = np.linalg.eigh(Bm)
    Bh = (V * np.sqrt(np.maximum(lam, 0.0))) @ V.T
    xb = truth[0] + Bh @ g.standard_normal(n_ADV)
    ys = []
    for t in range(OBS_T0, N_ADV + 1, OBS_TSTRIDE):
        pts = truth[t, ::OBS_STRIDE]
        ys.append(pts + SIG_O * g.standard_normal(pts.size))
    return truth, xb, np.concatenate(ys)


def advection_window(seed: int = 0, stream=None):
    """A library context holding the Section 5.1 window (propagator set
    through wc4d_set_propagator for every subwindow)."""
    import torch

    from . import (CORR_SOAR, MODEL_DENSE, Problem, wc4d_create, wc4d_set_background_obs, wc4d_set_covariance,
                   wc4d_set_propagator)
    prob = Problem()
    prob.n, prob.N, prob.model, prob.steps = n_ADV, N_ADV, MODEL_DENSE, 1
    prob.dt, prob.F, prob.sigma_o2 = 1.0 / N_ADV, 0.0, SIG_O ** 2
    prob.obs_stride, prob.obs_t0, prob.obs_tstride = OBS_STRIDE, OBS_T0, OBS_TSTRIDE
    prob.M_shared = 1
    ctx = wc4d_create(prob, stream)
    wc4d_set_covariance(ctx, 0, CORR_SOAR, SIG_B ** 2, LEN)
    wc4d_set_covariance(ctx, 1, CORR_SOAR, SIG_Q ** 2, LEN)
    M = torch.as_tensor(upwind_propagator(), dtype=torch.float64, device="cuda").contiguous()
    wc4d_set_propagator(ctx, -1, M)
    _, xb, y = advection_twin(seed)
    wc4d_set_background_obs(ctx, xb, y)
    return ctx


def dense_A(ctx, nA: int, block: int = 256) -> np.ndarray:
    """A (nA x nA) from FP64 block Hessian products with identity columns."""
    import torch

    from . import FP64, wc4d_hvp
    A = np.zeros((nA, nA))
    for j0 in range(0, nA, block):
        K = min(block, nA - j0)
        X = torch.zeros(K, nA, dtype=torch.float64, device="cuda")
        X[torch.arange(K), torch.arange(j0, j0 + K)] = 1.0
        Y = torch.zeros_like(X)
        wc4d_hvp(ctx, X, Y, K, nA, FP64)
        A[:, j0:j0 + K] = Y.cpu().numpy().T
    return A


def spectral_study(k: int = 25, l: int = 5, seeds=(0, 1, 2), ctx=None):
    """Section 5.1's comparison: Ritz values of REVD (Alg. 3), Nystrom (Alg. 4)
    and REVD_ritzit (Alg. 5) against A's exact eigenvalues, and the largest
    and smallest eigenvalues of the split-preconditioned C^T A C with each
    spectral LMP (eq. 16), averaged over probe seeds."""
    import torch

    from . import FP64, METHODS, wc4d_destroy, wc4d_get_ritz, wc4d_sketch
    own = ctx is None
    if own:
        ctx = advection_window()
    nA = n_ADV * (N_ADV + 1)
    A = dense_A(ctx, nA)
    A = 0.5 * (A + A.T)
    lam = np.sort(np.linalg.eigvalsh(A))[::-1]
    out = {"nA": nA, "nobs": int(10 * 10), "A_lambda_max": float(lam[0]), "A_lambda_min": float(lam[-1]),
           "A_eigenvalues_above_one": int(np.sum(lam > 1.0 + 1e-8)), "methods": {}}
    for name in ("revd", "nystrom", "ritzit"):
        errs5, errs, mx, mn = [], [], [], []
        for s in seeds:
            wc4d_sketch(ctx, METHODS[name], k, l, 0, 100 + s, None, FP64)
            U = torch.zeros(k, nA, dtype=torch.float64, device="cuda")
            th = wc4d_get_ritz(ctx, U, k)
            Uh = U.cpu().numpy()
            rel = np.abs(th - lam[:k]) / lam[:k]
            errs5.append(rel[:5].max())
            errs.append(rel.max())
            c = np.where(th > 0, 1.0 - 1.0 / np.sqrt(np.maximum(th, 1e-300)), 0.0)
            Cm = np.eye(nA) - (Uh.T * c) @ Uh
            ev = np.linalg.eigvalsh(Cm @ A @ Cm)
            mx.append(ev[-1])
            mn.append(ev[0])
        out["methods"][name] = {"ritz_max_rel_err_top5": float(np.mean(errs5)),
                                "ritz_max_rel_err_topk": float(np.mean(errs)),
                                "CAC_lambda_max": float(np.mean(mx)), "CAC_lambda_min": float(np.mean(mn)),
                                "CAC_condition": float(np.mean(np.array(mx) / np.array(mn)))}
    m = out["methods"]
    out["paper_claims"] = {
        "ritzit_worst_largest_ritz_values": m["ritzit"]["ritz_max_rel_err_topk"] >= max(
            m["revd"]["ritz_max_rel_err_topk"], m["nystrom"]["ritz_max_rel_err_topk"]),
        "preconditioned_lambda_max_below_A": all(v["CAC_lambda_max"] < lam[0] for v in m.values()),
        "revd_lambda_min_below_one": m["revd"]["CAC_lambda_min"] < 1.0 - 1e-6,
        "revd_condition_highest": m["revd"]["CAC_condition"] >= max(m["nystrom"]["CAC_condition"],
                                                                    m["ritzit"]["CAC_condition"]),
    }
    if own:
        wc4d_destroy(ctx)
    return out


# ---------------------------------------------------------------------------
# Section 5.2: Lorenz-96, n = 80, N = 150 one-step subwindows of an RK4 step
# of 0.025, every 10th variable observed at every 10th step (t = 10, .., 150:
# 120 observations), sigma_o = 0.15, B = 0.2^2 SOAR(2 dX), Q_t = 0.1^2 C_q with
# length 2 dX (SOAR standing in for the undefined Laplacian correlation).
# Inner loop 1 runs CG without a second-level preconditioner and keeps its
# Lanczos data; the second inner loop compares, over the same PCG iterations,
# no LMP, the deterministic LMP (Ritz pairs of inner loop 1, Section 3.3)
# and the randomised LMPs of REVD, Nystrom and REVD_ritzit (k = 5, l = 5).
# ---------------------------------------------------------------------------
L96_n, L96_N, L96_DT, L96_F = 80, 150, 0.025, 8.0
L96_SIG_O, L96_SIG_B, L96_SIG_Q, L96_LEN = 0.15, 0.2, 0.1, 2.0
L96_OBS = 10


def _l96_rhs(x, F=L96_F):
    return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F


def _l96_rk4(x, dt=L96_DT):
    k1 = _l96_rhs(x)
    k2 = _l96_rhs(x + 0.5 * dt * k1)
    k3 = _l96_rhs(x + 0.5 * dt * k2)
    k4 = _l96_rhs(x + dt * k3)
    return x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


def lorenz96_twin(seed: int = 0, spinup_steps: int = 2000, obs: int = L96_OBS):
    """Truth (N + 1, n) after an RK4 spin-up from x = F (+ 0.01 noise),
    background truth + B^{1/2} noise, observations of every `obs`-th
    variable at every `obs`-th step (obs = 10: 120, 5: 480, 2: 3000)."""
    g = np.random.default_rng([int(seed), 52])
    x = L96_F + 0.01 * g.standard_normal(L96_n)
    for _ in range(spinup_steps):
        x = _l96_rk4(x)
    truth = np.zeros((L96_N + 1, L96_n))
    truth[0] = x
    for t in range(L96_N):
        truth[t + 1] = _l96_rk4(truth[t])
    row = soar_row(L96_n, L96_SIG_B ** 2, L96_LEN)
    Bm = np.array([np.roll(row, i) for i in range(L96_n)])
    lam, V = np.linalg.eigh(Bm)
    Bh = (V * np.sqrt(np.maximum(lam, 0.0))) @ V.T
    xb = truth[0] + Bh @ g.standard_normal(L96_n)
    ys = []
    for t in range(obs, L96_N + 1, obs):
        pts = truth[t, ::obs]
        ys.append(pts + L96_SIG_O * g.standard_normal(pts.size))
    return truth, xb, np.concatenate(ys)


def lorenz96_window(seed: int = 0, stream=None, obs: int = L96_OBS):
    from . import (CORR_SOAR, MODEL_L96, Problem, wc4d_create, wc4d_set_background_obs, wc4d_set_covariance)
    prob = Problem()
    prob.n, prob.N, prob.model, prob.steps = L96_n, L96_N, MODEL_L96, 1
    prob.dt, prob.F, prob.sigma_o2 = L96_DT, L96_F, L96_SIG_O ** 2
    prob.obs_stride, prob.obs_t0, prob.obs_tstride = obs, obs, obs
    prob.M_shared = 0
    ctx = wc4d_create(prob, stream)
    wc4d_set_covariance(ctx, 0, CORR_SOAR, L96_SIG_B ** 2, L96_LEN)
    wc4d_set_covariance(ctx, 1, CORR_SOAR, L96_SIG_Q ** 2, L96_LEN)
    _, xb, y = lorenz96_twin(seed, obs=obs)
    wc4d_set_background_obs(ctx, xb, y)
    return ctx


def _lambda_min_CAC(ctx, nA, nobs, U, theta, seed=0):
    """Smallest eigenvalue of C^T A C for the spectral LMP C = I - U diag(c)
    U^T (c = 1 - theta^{-1/2}).  A - I has rank <= q (eq. 10) and C - I rank
    <= k, so every eigenvector outside V = range(A - I) + range(U) has
    eigenvalue 1 and V is invariant: the eigenvalues of Q^T C A C Q, Q an
    orthonormal basis of V (from (A - I) G with q + 10 Gaussian columns and
    U), are the rest.  Products with A: FP64 block Hessian products."""
    import torch

    from . import FP64, wc4d_hvp
    g = np.random.default_rng(seed)
    m = nobs + 10
    G = torch.as_tensor(g.standard_normal((m, nA)), device="cuda")
    Y = torch.zeros_like(G)
    wc4d_hvp(ctx, G, Y, m, nA, FP64)
    R = (Y - G).cpu().numpy()                        # rows span range(A - I)
    Q, _ = np.linalg.qr(np.vstack([R, U]).T)         # nA x r
    c = np.where(theta > 0, 1.0 - 1.0 / np.sqrt(np.maximum(theta, 1e-300)), 0.0)

    def C(X):                                        # X: nA x r
        return X - U.T @ (c[:, None] * (U @ X))

    CQ = C(Q)
    Xd = torch.as_tensor(np.ascontiguousarray(CQ.T), device="cuda")
    Yd = torch.zeros_like(Xd)
    wc4d_hvp(ctx, Xd, Yd, Xd.shape[0], nA, FP64)
    CACQ = C(Yd.cpu().numpy().T)
    S = Q.T @ CACQ
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    return float(min(ev.min(), 1.0)) if Q.shape[1] < nA else float(ev.min())


def lorenz96_study(k: int = 5, l: int = 5, iters: int = 10, seeds=(0, 1, 2), window_seed: int = 0,
                   obs: int = L96_OBS, k_det=None, lmin: bool = True):
    """Section 5.2's comparison in the second inner loop: the quadratic-cost
    decrease after each of `iters` PCG iterations (FP64) with no LMP, the
    deterministic LMP (k_det Ritz pairs of inner loop 1, default k) and the
    three randomised LMPs (k pairs, l oversampling; averaged over probe
    seeds), and (lmin) the smallest eigenvalue of C^T A C for each LMP.  obs:
    the observation network (every obs-th variable at every obs-th step)."""
    import torch

    from . import (FP64, METHODS, wc4d_destroy, wc4d_get_ritz, wc4d_lanczos_cg, wc4d_lanczos_ritz, wc4d_nobs,
                   wc4d_outer_update, wc4d_pcg, wc4d_set_ritz, wc4d_sketch)
    k_det = k if k_det is None else k_det
    ctx = lorenz96_window(window_seed, obs=obs)
    nA = L96_n * (L96_N + 1)
    nobs = int(wc4d_nobs(ctx))
    x = torch.zeros(nA, dtype=torch.float64, device="cuda")
    J, rr1 = wc4d_lanczos_cg(ctx, x, 1e-6, 100, reorth=True)          # inner loop 1, no LMP
    wc4d_lanczos_ritz(ctx, k_det)
    Ud = torch.zeros(k_det, nA, dtype=torch.float64, device="cuda")
    thd = wc4d_get_ritz(ctx, Ud, k_det)
    wc4d_outer_update(ctx, x)                                          # second linearisation
    out = {"nA": nA, "nobs": nobs, "inner_loop_1": {"cg_iters": J, "relres": rr1}, "k": k, "l": l,
           "k_deterministic": k_det, "qcf_decrease": {}, "lambda_min_CAC": {}}
    y = torch.zeros(nA, dtype=torch.float64, device="cuda")

    def qcf_curve(use):
        _, _, drop, _ = wc4d_pcg(ctx, y, 1e-14, iters, use, iters, FP64, qcf=True, raise_on_noconv=False)
        return np.cumsum(drop)

    wc4d_set_ritz(ctx, 0, None, np.zeros(0))
    out["qcf_decrease"]["none"] = qcf_curve(0).tolist()
    wc4d_set_ritz(ctx, k_det, Ud, thd)
    out["qcf_decrease"]["deterministic"] = qcf_curve(1).tolist()
    if lmin:
        out["lambda_min_CAC"]["deterministic"] = _lambda_min_CAC(ctx, nA, nobs, Ud.cpu().numpy(), thd)
    for name in ("revd", "nystrom", "ritzit"):
        curves, lmins = [], []
        for s in seeds:
            th = wc4d_sketch(ctx, METHODS[name], k, l, 0, 200 + s, None, FP64)
            curves.append(qcf_curve(1))
            if lmin:
                U = torch.zeros(k, nA, dtype=torch.float64, device="cuda")
                th = wc4d_get_ritz(ctx, U, k)
                lmins.append(_lambda_min_CAC(ctx, nA, nobs, U.cpu().numpy(), th))
        out["qcf_decrease"][name] = np.mean(curves, axis=0).tolist()
        if lmin:
            out["lambda_min_CAC"][name] = float(np.mean(lmins))
    q = {m: v[-1] for m, v in out["qcf_decrease"].items()}
    out["paper_claims"] = {
        "randomised_beat_deterministic": all(q[m] > q["deterministic"] for m in ("revd", "nystrom", "ritzit")),
        "ritzit_best": q["ritzit"] >= max(q["revd"], q["nystrom"]),
    }
    if lmin:
        out["paper_claims"]["revd_lambda_min_below_nystrom_ritzit"] = out["lambda_min_CAC"]["revd"] < min(
            out["lambda_min_CAC"]["nystrom"], out["lambda_min_CAC"]["ritzit"])
    wc4d_destroy(ctx)
    return out


def lorenz96_networks(networks=(5, 2), ks=(5, 15), l: int = 5, iters: int = 10, seeds=(0, 1, 2)):
    """Section 5.2's denser observation networks: every 5th variable at every
    5th step (480 observations) and every 2nd at every 2nd step (3000), each
    with k = 5 and k = 15 (l = 5), plus the randomised LMPs with k = 5 against
    the deterministic LMP with k = 15.  Reported per network and k: the
    quadratic-cost decrease after `iters` PCG iterations of each LMP, and the
    spread of the three randomised LMPs relative to their mean (the paper:
    little difference between them when k is small relative to q)."""
    out = {}
    for obs in networks:
        rows = {}
        for k in ks:
            r = lorenz96_study(k=k, l=l, iters=iters, seeds=seeds, obs=obs, lmin=False)
            q = {m: v[-1] for m, v in r["qcf_decrease"].items()}
            rnd = [q["revd"], q["nystrom"], q["ritzit"]]
            rows[f"k{k}"] = {"nobs": r["nobs"], "qcf_final": q,
                             "randomised_spread": (max(rnd) - min(rnd)) / float(np.mean(rnd)),
                             "randomised_beat_deterministic": r["paper_claims"]["randomised_beat_deterministic"]}
        # randomised LMPs with k = 5 against the deterministic LMP with k = 15
        r = lorenz96_study(k=min(ks), l=l, iters=iters, seeds=seeds, obs=obs, k_det=max(ks), lmin=False)
        q = {m: v[-1] for m, v in r["qcf_decrease"].items()}
        rows[f"randomised_k{min(ks)}_vs_deterministic_k{max(ks)}"] = {
            "qcf_final": q, "randomised_beat_deterministic": r["paper_claims"]["randomised_beat_deterministic"]}
        out[f"q{rows[f'k{min(ks)}']['nobs']}"] = rows
    return out
