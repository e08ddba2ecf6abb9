"""Surrogate workflow: trajectories from the solver, FNO training with the
library's kernels, and surrogate-assisted integration with the integrator as
verifier.

Everything numerical runs in libpf.so; this module only orchestrates calls.
Training data are pairs (y(t), y(t + tau)) of real-space states taken every
tau along trajectories integrated with fixed ARK4 steps of size dt
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


def train(net, traj, epochs, lr, seed=0, log=None):
    """Adam, one snapshot pair per step, on the MSE of normalised increments
    over all consecutive snapshot pairs of a CUDA float32 trajectory tensor
    [n, T, 4, ...]; the normalisation statistics and every per-pair
    transformation are computed by the library.  Returns the per-epoch mean
    losses."""
    net.fit_norm(traj)
    n, T = traj.shape[0], traj.shape[1] - 1
    pairs = [(i, t) for i in range(n) for t in range(T)]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(len(pairs))
        tot = 0.0
        for k in order:
            i, t = pairs[k]
            tot += net.train_pair(traj[i, t], traj[i, t + 1], lr)
        losses.append(tot / len(pairs))
        if log:
            log("epoch %d loss %.4e" % (ep, losses[-1]))
    return losses


def rollout(y0, params, t_end, tau, net=None, precision="fp32bulk", rtol=1e-4, atol=1e-8, h0=1.0):
    """Integrate to t_end adaptively (ARK4, rtol/atol).  Without a network:
    one pf_advance.  With a network: window by window of length tau, each
    window first proposed by the network and then integrated by the method,
    which checks the proposal (accepted when its WRMS distance to the
    verified state is <= 1); the state always continues from the verified
    integration.  Returns (final real-space state, wall seconds, accepted,
    offered, proposal distances)."""
    import torch
    shape = y0.shape[1:]
    acc = off = 0
    dists = []
    with Simulation(shape, params, "ark4", precision) as s:
        s.set_state(y0)
        s.set_time(0.0, h0)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        if net is None:
            s.advance(t_end, rtol, atol)
        else:
            t = 0.0
            while t < t_end - 1e-9:
                w = min(tau, t_end - t)
                off += 1
                ok, d = net.surrogate_step(s, w, h0, rtol, atol)
                acc += int(ok)
                dists.append(d)
                t = s.time()[0]
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        out = s.get_state()
    return out, wall, acc, off, dists


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
