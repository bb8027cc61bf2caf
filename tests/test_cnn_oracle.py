"""Pins of the CNN oracle (FP64): its forward equals torch's CPU conv1d chain
(float64, an independent library routine) and its hand-written gradient equals
central finite differences of its loss."""
import numpy as np
import pytest

from oracle import cnn


def test_param_count():
    assert cnn.n_params() == 9328


def test_forward_matches_torch_conv1d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p = cnn.init_params(3) + 0.05 * rng.standard_normal(cnn.n_params())
    x = rng.standard_normal((57, 16))
    y = cnn.forward_member(x, p)
    a = torch.tensor(x.T[None], dtype=torch.float64)
    for (W, b, relu), (ci, co, _) in zip(cnn.unpack(p), cnn.LAYERS):
        w = torch.tensor(W.reshape(co, 3, ci).transpose(0, 2, 1).copy(), dtype=torch.float64)
        a = torch.nn.functional.conv1d(a, w, torch.tensor(b), padding=1)
        if relu:
            a = torch.relu(a)
    assert np.allclose(y, a[0, 0].numpy(), rtol=1e-12, atol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = cnn.init_params(4) + 0.05 * rng.standard_normal(cnn.n_params())
    xs = [rng.standard_normal((23, 16)), rng.standard_normal((9, 16))]
    ts = [rng.standard_normal(23), rng.standard_normal(9)]
    ms = [(rng.random(23) < 0.7).astype(float), np.ones(9)]
    L, g = cnn.loss_and_grad(xs, p, ts, ms)
    idx = rng.choice(cnn.n_params(), size=60, replace=False)
    idx = np.concatenate([idx, [0, 1535, 1536 + 32, cnn.n_params() - 17, cnn.n_params() - 1]])
    eps = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += eps
        Lp, _ = cnn.loss_and_grad(xs, q, ts, ms)
        q[i] -= 2 * eps
        Lm, _ = cnn.loss_and_grad(xs, q, ts, ms)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
