"""FP64 CPU oracle of the learned initial-guess network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the plain definition the
GPU's BF16 tensor-core kernels are checked against.

Network: four 1D convolutions of width 3 over the cells of each member, zero
padding outside the member's cells; channels 16 -> 32 -> 32 -> 32 -> 16, ReLU
after the first three, output = channel 0 of the last layer (the other 15
output channels pad the last GEMM to the tensor-core N granularity and are
unused).  Parameters are one flat FP32 vector, per layer W[c_out][3 c_in] then
b[c_out], with W's column k * c_in + c weighting input channel c of the cell
at offset k - 1.

Loss: L = sum(mask (y - t)^2) / max(1, sum(mask)).
"""
from __future__ import annotations

import numpy as np

LAYERS = ((16, 32, True), (32, 32, True), (32, 32, True), (32, 16, False))


def n_params() -> int:
    return sum(co * 3 * ci + co for ci, co, _ in LAYERS)


def unpack(params):
    params = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for ci, co, relu in LAYERS:
        W = params[o:o + co * 3 * ci].reshape(co, 3 * ci)
        o += co * 3 * ci
        b = params[o:o + co]
        o += co
        out.append((W, b, relu))
    assert o == params.size
    return out


def _shifted(a):
    """(n, c) -> (n, 3c): row i = [a[i-1], a[i], a[i+1]] with zeros outside."""
    n, c = a.shape
    z = np.zeros((1, c))
    left = np.vstack([z, a[:-1]])
    right = np.vstack([a[1:], z])
    return np.hstack([left, a, right])


def forward_member(x, params, keep=False):
    """x: (nx, 16) features of one member -> y (nx,), [activations]."""
    acts = [np.asarray(x, dtype=np.float64)]
    a = acts[0]
    for W, b, relu in unpack(params):
        z = _shifted(a) @ W.T + b
        a = np.maximum(z, 0.0) if relu else z
        acts.append(a)
    return (a[:, 0], acts) if keep else a[:, 0]


def loss_and_grad_member(x, params, t, mask):
    """Loss contribution (un-normalised sum) and gradient of one member."""
    y, acts = forward_member(x, params, keep=True)
    m = np.asarray(mask, dtype=np.float64)
    r = (y - t) * m
    loss = float(np.sum(r * (y - t)))
    layers = unpack(params)
    grads = []
    nx = y.size
    d = np.zeros((nx, layers[-1][0].shape[0]))
    d[:, 0] = 2.0 * r                       # dL/dz of the last (linear) layer
    for li in range(len(layers) - 1, -1, -1):
        W, b, relu = layers[li]
        a_in = acts[li]
        if relu:
            d = d * (acts[li + 1] > 0.0)
        grads.append((d.T @ _shifted(a_in), d.sum(axis=0)))
        # back through the convolution: dA[i] = sum_k d[i - k + 1] W[:, k-block]
        ci = a_in.shape[1]
        dS = d @ W                           # (nx, 3 ci): gradient w.r.t. shifted rows
        da = dS[:, ci:2 * ci].copy()
        da[1:] += dS[:-1, 2 * ci:]           # row i used as the right neighbour of row i-1
        da[:-1] += dS[1:, :ci]               # row i used as the left neighbour of row i+1
        d = da
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat


def loss_and_grad(xs, params, ts, masks):
    """Over members (lists): normalised loss and gradient."""
    tot, g, cnt = 0.0, np.zeros(n_params()), 0.0
    for x, t, m in zip(xs, ts, masks):
        l, gr = loss_and_grad_member(x, params, t, m)
        tot += l
        g += gr
        cnt += float(np.sum(m))
    den = max(1.0, cnt)
    return tot / den, g / den


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for ci, co, _ in LAYERS:
        out.append(rng.normal(0.0, np.sqrt(2.0 / (3 * ci)), size=co * 3 * ci))
        out.append(np.zeros(co))
    return np.concatenate(out)
