"""Trains the learned sketch proposal (the 4-layer periodic 1D convolutional
encoder that `wc4d_learned_probes` runs) and writes its BF16 weights.

Targets: the top-64 Ritz vectors that the library's own randomised EVD
(REVD, q = 1, 64 + 32 Gaussian probes) produces for seeded Lorenz-96 windows
(n = 8192, N = 10 subwindows of 8 RK4 steps; seeds 20000 + i).  The Hessian
depends on the background (the linearisation trajectory) and the observation
network, not on the observed values, so a training window needs only a
background: a state spun up on the attractor by RK4 (5 time units from
F + 0.01 N(0, 1)) plus a smooth random field of the background-error
covariance's length and variance, as in the synthetic twin.  Loss: one minus
the captured fraction ||U^T orth(S)||_F^2 / 64 of the target subspace.
Training uses PyTorch's autograd (offline; the inference on the hot path runs
in the library's kernels).

    python -m paper_2101_07249_gb300.learned.train --count 2000 --epochs 8
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "l96_n8192_N10_m64.npz")


def window(seed):
    from paper_2101_07249_gb300 import inputs
    return inputs.L96.replace(N=10, name=f"l96_n8192_N10_s{seed}", seed=seed, k=64, l=32)


def rk4_boundaries(x0, F, dt, N, steps):
    """States at the subwindow boundaries of the unforced RK4 run."""
    def f(x):
        return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F
    out = [np.array(x0, dtype=np.float64)]
    x = out[0].copy()
    for _ in range(N):
        for _ in range(steps):
            k1 = f(x); k2 = f(x + 0.5 * dt * k1); k3 = f(x + 0.5 * dt * k2); k4 = f(x + dt * k3)
            x = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        out.append(x.copy())
    return np.array(out)


def rk4_run(x0, F, dt, nsteps):
    def f(x):
        return (np.roll(x, -1) - np.roll(x, 2)) * np.roll(x, 1) - x + F
    x = np.array(x0, dtype=np.float64)
    for _ in range(nsteps):
        k1 = f(x); k2 = f(x + 0.5 * dt * k1); k3 = f(x + 0.5 * dt * k2); k4 = f(x + dt * k3)
        x = x + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


def background(cfg, spinup=5.0):
    """A training window's background: an RK4 spin-up onto the attractor plus
    a smooth field of variance b_var and length b_L (the twin's recipe)."""
    from paper_2101_07249_gb300 import inputs
    g = inputs.rng(cfg.seed, 1)
    x0 = cfg.F + 0.01 * g.standard_normal(cfg.n)
    xs = rk4_run(x0, cfg.F, cfg.dt, int(round(spinup / cfg.dt)))
    return xs + inputs._smooth_field(g, cfg.n, cfg.b_L, cfg.b_var)


def features(cfg, xb):
    traj = rk4_boundaries(xb, cfg.F, cfg.dt, cfg.N, cfg.steps) / cfg.F
    mask = np.zeros((cfg.N + 1, cfg.n))
    for t in range(cfg.obs_t0, cfg.N + 1):
        mask[t, ::cfg.obs_stride] = 1.0
    return np.concatenate([traj, mask]).astype(np.float32)


def make_net(N, m):
    import torch.nn as nn
    c0 = 2 * (N + 1)
    return nn.Sequential(
        nn.Conv1d(c0, 64, 5, padding=2, padding_mode="circular"), nn.ReLU(),
        nn.Conv1d(64, 64, 5, padding=2, padding_mode="circular"), nn.ReLU(),
        nn.Conv1d(64, 64, 5, padding=2, padding_mode="circular"), nn.ReLU(),
        nn.Conv1d(64, m * (N + 1), 1))


def captured(net, x, U, m, Np1):
    """Fraction of the target subspace (rows of U, orthonormal) captured by
    the span of the network's m columns."""
    import torch
    S = net(x[None])[0].reshape(m, Np1, -1).reshape(m, -1)
    Q, _ = torch.linalg.qr(S.T)
    return (U @ Q).square().sum() / U.shape[0]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--holdout", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()

    import torch
    import paper_2101_07249_gb300 as w
    from paper_2101_07249_gb300 import inputs

    m = 64
    data = []
    t0 = time.time()
    for i in range(args.count + args.holdout):
        cfg = window(20000 + i)
        xb = background(cfg)
        S = w.Solver(cfg)
        w.wc4d_set_background_obs(S.ctx, xb, np.zeros(cfg.nobs))
        w.wc4d_sketch(S.ctx, w.REVD, m, cfg.l, 1, 7 + i, None, w.MIXED)
        U = torch.zeros(m, cfg.nA, dtype=torch.float64, device="cuda")
        w.wc4d_get_ritz(S.ctx, U, m)
        S.close()
        data.append((torch.as_tensor(features(cfg, xb), device="cuda"), U.float()))
        if (i + 1) % 250 == 0:
            print(f"  {i + 1} windows, {time.time() - t0:.0f} s", flush=True)
    print(f"targets: {len(data)} windows in {time.time() - t0:.0f} s", flush=True)

    cfg = window(0)
    Np1 = cfg.N + 1
    torch.manual_seed(0)
    net = make_net(cfg.N, m).cuda()
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    train, held = data[:args.count], data[args.count:]
    for ep in range(args.epochs):
        perm = torch.randperm(len(train)).tolist()
        tot = 0.0
        for j in perm:
            x, U = train[j]
            loss = 1.0 - captured(net, x, U, m, Np1)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach())
        with torch.no_grad():
            hv = float(np.mean([float(captured(net, x, U, m, Np1)) for x, U in held]))
        print(f"epoch {ep}: train loss {tot / len(train):.4f}  held-out captured {hv:.4f}", flush=True)

    with torch.no_grad():
        gauss = float(np.mean([float((U @ torch.linalg.qr(torch.randn(cfg.nA, m, device='cuda'))[0]).square().sum()
                                     / m) for _, U in held]))
    convs = [mod for mod in net if isinstance(mod, torch.nn.Conv1d)]
    bits, biases = [], []
    for cv in convs:
        Wf = cv.weight.detach().float().cpu().numpy()
        u = Wf.view(np.uint32).astype(np.uint64)
        rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)   # round to nearest even
        bits.append(rounded)
        biases.append(cv.bias.detach().float().cpu().numpy())
    np.savez(args.out, W0=bits[0], W1=bits[1], W2=bits[2], W3=bits[3], b0=biases[0], b1=biases[1],
             b2=biases[2], b3=biases[3], n=cfg.n, N=cfg.N, m=m, held_out_captured=hv, gaussian_captured=gauss)
    print(f"wrote {args.out}: held-out captured {hv:.4f} (a Gaussian block of {m}: {gauss:.4f})", flush=True)


if __name__ == "__main__":
    main()
