"""Training the learned initial guess on pairs the method generates.

Host orchestration only: every forward, backward and Adam update runs in the
CUDA library (``nh_cnn_loss_grad``, ``nh_cnn_adam``); this module draws
minibatches and keeps the tensors.

Typical use::

    G = grid_from_workload(wl); G.cnn_attach(); G.cnn_record(True)
    samples = collect(G, dt, 120)            # plain method, harvested each step
    params, losses = train(samples)          # GPU kernels
    G.cnn_set_params(params); G.set_solver(guess=NH_GUESS_CNN)
"""
from __future__ import annotations

import numpy as np

from . import nhswe as N

# (c_in, c_out) of the four layers, in parameter order (see nhswe_cnn.h)
LAYERS = ((16, 32), (32, 32), (32, 32), (32, 16))


def init_params(seed=0, last_gain=0.01):
    """He-normal weights, zero biases, as a CUDA float32 tensor.  The last
    layer is scaled by ``last_gain`` so that an untrained network adds almost
    nothing to the quadratic extrapolation it corrects."""
    import torch
    rng = np.random.default_rng(seed)
    out = []
    for k, (ci, co) in enumerate(LAYERS):
        w = rng.normal(0.0, np.sqrt(2.0 / (3 * ci)), size=co * 3 * ci)
        if k == len(LAYERS) - 1:
            w *= last_gain
        out += [w, np.zeros(co)]
    p = np.concatenate(out)
    assert p.size == N.NH_CNN_PARAMS
    return torch.tensor(p, dtype=torch.float32, device="cuda")


def collect(G, dt, n_steps, samples=None):
    """Run ``n_steps`` steps in record mode and harvest each: appends
    (features, target, mask, cells per member) for every step with at least
    one target cell, and returns the list."""
    G.cnn_record(True)
    out = [] if samples is None else samples
    nxd = G.nx_device()
    for _ in range(n_steps):
        G.step(dt)
        f, t, m, s = G.cnn_harvest()
        if s > 0.0 and int(m.count_nonzero().item()) > 0:
            out.append((f, t, m, nxd))
    return out


def train(samples, steps=600, lr=2e-3, batch=16, seed=0, params=None):
    """Adam on the harvested pairs, minibatches of member rows drawn
    uniformly.  Returns (params, per-step losses)."""
    import torch
    if not samples:
        raise ValueError("no training samples")
    feats = torch.cat([s[0] for s in samples])
    tgts = torch.cat([s[1] for s in samples])
    msks = torch.cat([s[2] for s in samples])
    nxs = torch.cat([s[3] for s in samples])
    rows, pitch = tgts.shape
    batch = min(batch, rows)
    p = init_params(seed) if params is None else params.clone()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    g = torch.zeros_like(p)
    ws = N.CnnWorkspace(batch, pitch)
    gen = torch.Generator().manual_seed(seed)
    losses = []
    for k in range(1, steps + 1):
        idx = torch.randint(0, rows, (batch,), generator=gen).cuda()
        losses.append(N.nh_cnn_loss_grad(feats[idx].contiguous(), nxs[idx].contiguous(), p, tgts[idx].contiguous(),
                                         msks[idx].contiguous(), g, ws))
        N.nh_cnn_adam(p, g, m, v, k, lr)
    return p, losses
