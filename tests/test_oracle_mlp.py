"""Pins of the FP64 proposer MLP reference (CPU)."""

import numpy as np
import pytest

from oracle import mlp
from paper_2402_02585_gb300 import instances

DIMS = (10, 16, 6)


def _data(B=7, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, DIMS[0]))
    y = rng.uniform(0, 2 * np.pi, size=(B, DIMS[2]))
    params = instances.random_mlp_params(*DIMS, seed=seed).astype(np.float64)
    params += 0.01 * rng.normal(size=params.shape)  # nonzero biases too
    return params, x, y


def test_gelu_identities():
    x = np.linspace(-6, 6, 101)
    assert abs(mlp.gelu(np.array([0.0]))[0]) == 0.0
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-14)
    assert np.allclose(mlp.gelu(np.array([10.0, -10.0])), [10.0, 0.0], atol=1e-12)
    h = 1e-6
    assert np.allclose((mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), mlp.gelu_grad(x), atol=1e-8)


def test_forward_and_grad_match_torch_float64():
    torch = pytest.importorskip("torch")
    params, x, y = _data()
    d_in, d_h, d_out = DIMS
    ang, _ = mlp.forward(params, x, DIMS)
    loss, g = mlp.loss_and_grad(params, x, y, DIMS)
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    o = 0
    parts = []
    for s in (d_h * d_in, d_h, d_h * d_h, d_h, d_out * d_h, d_out):
        parts.append(P[o:o + s])
        o += s
    W1, b1, W2, b2, W3, b3 = parts
    X = torch.tensor(x)
    h1 = torch.nn.functional.gelu(torch.nn.functional.linear(X, W1.view(d_h, d_in), b1))
    h2 = torch.nn.functional.gelu(torch.nn.functional.linear(h1, W2.view(d_h, d_h), b2))
    a = 2 * np.pi * torch.sigmoid(torch.nn.functional.linear(h2, W3.view(d_out, d_h), b3))
    L = torch.mean(2 * (1 - torch.cos(a - torch.tensor(y))))
    L.backward()
    assert np.allclose(ang, a.detach().numpy(), atol=1e-12)
    assert abs(loss - L.item()) < 1e-12
    assert np.allclose(g, P.grad.numpy(), atol=1e-12)


def test_grad_matches_finite_differences():
    params, x, y = _data(seed=3)
    _, g = mlp.loss_and_grad(params, x, y, DIMS)
    rng = np.random.default_rng(1)
    h = 1e-6
    for i in rng.choice(len(params), 25, replace=False):
        pp = params.copy()
        pp[i] += h
        up, _ = mlp.loss_and_grad(pp, x, y, DIMS)
        pp[i] -= 2 * h
        dn, _ = mlp.loss_and_grad(pp, x, y, DIMS)
        assert abs((up - dn) / (2 * h) - g[i]) < 1e-7


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    p0 = np.zeros(4)
    p1, m, v = mlp.adam(p0, g, np.zeros(4), np.zeros(4), t=1, lr=0.01, eps=0.0)
    assert np.allclose(p1, -0.01 * np.sign(g), atol=1e-15)


def test_features_layout():
    x = mlp.features([2, 3, 1], n=2, m=2, d_in=8)
    assert np.allclose(x, [0.5, 0.75, 0.25, 0, 0, 0, 2 / 32, 2 / 128])


def test_loss_is_periodic_and_quadratic_near_zero():
    params, x, y = _data(B=3, seed=4)
    ang, _ = mlp.forward(params, x, DIMS)
    l0, _ = mlp.loss_and_grad(params, x, ang, DIMS)
    assert abs(l0) < 1e-15
    l1, _ = mlp.loss_and_grad(params, x, ang + 2 * np.pi, DIMS)
    assert abs(l1) < 1e-12
    d = 1e-3
    l2, _ = mlp.loss_and_grad(params, x, ang + d, DIMS)
    assert abs(l2 - d * d) < 1e-12
