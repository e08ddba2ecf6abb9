"""Surrogate workflow: trajectories from the solver, FNO training with the
library's kernels, and surrogate-assisted integration with the integrator as
judge.

Everything numerical runs in libpf.so; this module only orchestrates calls.
Training data are pairs (y(t), y(t + tau) - y(t)) of real-space states taken
every tau along trajectories integrated with fixed ARK4 steps of size dt
(tau = 8 dt).
"""
from __future__ import annotations

import time

import numpy as np

from . import FNO, Simulation


def trajectories(ics, params, dt, n_snap, steps_per_snap=8, precision="fp32bulk"):
    """Integrate each initial condition with fixed ARK4 steps and return the
    snapshots as a CUDA float32 tensor [n_traj, n_snap + 1, 4, nz, ny, nx]."""
    import torch
    out = []
    for y0, p in ics:
        shape = y0.shape[1:]
        snaps = []
        with Simulation(shape, p, "ark4", precision) as s:
            s.set_state(y0)
            buf = torch.empty((4,) + shape, dtype=torch.float64, device="cuda")
            s.get_state(buf)
            snaps.append(buf.float().clone())
            for _ in range(n_snap):
                for _ in range(steps_per_snap):
                    s.step(dt, want_lte=False)
                s.get_state(buf)
                snaps.append(buf.float().clone())
        out.append(torch.stack(snaps))
    return torch.stack(out)


def normalisation(traj):
    """Per-channel input mean/std and output (increment) std of a trajectory
    tensor [n, T, 4, ...]."""
    x = traj[:, :-1].transpose(0, 2).reshape(4, -1)
    dlt = (traj[:, 1:] - traj[:, :-1]).transpose(0, 2).reshape(4, -1)
    mean = x.mean(dim=1)
    std = x.std(dim=1).clamp_min(1e-6)
    dstd = dlt.std(dim=1).clamp_min(1e-9)
    return mean.cpu().numpy(), std.cpu().numpy(), dstd.cpu().numpy()


def train(net, traj, epochs, lr, seed=0, log=None):
    """Adam on the MSE of normalised increments over all consecutive snapshot
    pairs; returns the per-epoch mean losses."""
    import torch
    mean, std, dstd = normalisation(traj)
    net.set_norm(mean, std, dstd)
    m = torch.as_tensor(mean, device="cuda").view(4, 1, 1, 1)
    sd = torch.as_tensor(std, device="cuda").view(4, 1, 1, 1)
    ds = torch.as_tensor(dstd, device="cuda").view(4, 1, 1, 1)
    n, T = traj.shape[0], traj.shape[1] - 1
    pairs = [(i, t) for i in range(n) for t in range(T)]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for k in order:
            i, t = pairs[k]
            x = ((traj[i, t] - m) / sd).contiguous()
            y = ((traj[i, t + 1] - traj[i, t]) / ds).contiguous()
            tot += net.train_step(x, y, lr)
        losses.append(tot / len(pairs))
        if log:
            log("epoch %d loss %.4e" % (ep, losses[-1]))
    return losses


def rollout(y0, params, t_end, dt, net=None, steps_per_snap=8, precision="fp32bulk", rtol=1e-4, atol=1e-8):
    """Integrate to t_end with fixed ARK4 steps of size dt; with a network,
    each block of steps_per_snap steps is first offered to the surrogate
    (proposal over tau = steps_per_snap * dt plus one judged step of size dt).
    Returns (final real-space state, wall seconds, accepted, offered)."""
    import torch
    shape = y0.shape[1:]
    tau = steps_per_snap * dt
    acc = off = 0
    with Simulation(shape, params, "ark4", precision) as s:
        s.set_state(y0)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        t = 0.0
        while t < t_end - 1e-9:
            left = t_end - t
            if net is not None and left >= tau + dt - 1e-9:
                off += 1
                ok, _ = net.surrogate_step(s, tau, dt, rtol, atol)
                if ok:
                    acc += 1
                    t += tau + dt
                    continue
            k = min(steps_per_snap, int(round(left / dt)))
            for _ in range(max(k, 1)):
                s.step(dt, want_lte=False)
            t += max(k, 1) * dt
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        out = s.get_state()
    return out, wall, acc, off


def new_network(shape, C=32, modes=12, H=128, L=4, bf16=True, seed=0):
    """FNO with a seeded initialisation (uniform, fan-in scaled; spectral
    weights 1/C^2)."""
    net = FNO(shape, C=C, modes=modes, H=H, L=L, bf16=bf16)
    rng = np.random.default_rng(seed)
    theta = np.zeros(net.n, dtype=np.float32)
    # layout: P[C][4], p[C], per layer W (K C C 2), V (C C), v (C), Q1 (H C), q1, Q2 (4 H), q2
    K = 4 * modes ** 3
    o = 0

    def put(count, scale):
        nonlocal o
        theta[o:o + count] = rng.uniform(-1, 1, count) * scale
        o += count

    put(C * 4, 0.5)
    o += C
    for _ in range(L):
        put(K * C * C * 2, 1.0 / (C * C))
        put(C * C, 1.0 / np.sqrt(C))
        o += C
    put(H * C, 1.0 / np.sqrt(C))
    o += H
    put(4 * H, 1.0 / np.sqrt(H))
    o += 4
    assert o == net.n
    net.set_params(theta)
    return net
