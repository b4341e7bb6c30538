"""Pins for the FP64 MLP oracle: each one fails for a plausible slip (a dropped term in the
GELU derivative, a transposed weight gradient, a missing bias-correction in Adam)."""
import math

import numpy as np
import pytest
from scipy.special import erf

from oracle import mlp


def _params(sizes, seed):
    rng = np.random.default_rng(seed)
    return [(rng.normal(0, 1 / math.sqrt(i), (o, i)), rng.normal(0, 0.1, o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_gelu_identities_and_the_exact_gelu():
    x = np.linspace(-6, 6, 2001)
    # 0.5 x (1 + tanh u) - 0.5 (-x)(1 + tanh(-u)) = x for the tanh form (odd tanh)
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15, rtol=0)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    # the tanh form approximates x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)) to a few 1e-4
    exact = 0.5 * x * (1 + erf(x / math.sqrt(2)))
    assert np.max(np.abs(mlp.gelu(x) - exact)) < 1e-3
    assert abs(mlp.gelu(np.array([30.0]))[0] - 30.0) < 1e-12


def test_gelu_grad_matches_central_difference():
    x = np.linspace(-5, 5, 101)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-8


def test_single_linear_layer_has_the_closed_form_gradient():
    """No hidden layer: y = x W^T + b, loss mean (y - t)^2, so dL/dW = 2/(B n) (y - t)^T x and
    dL/db = 2/(B n) sum_rows (y - t), written out element by element."""
    rng = np.random.default_rng(1)
    B, k, n = 7, 5, 3
    W, b = rng.normal(size=(n, k)), rng.normal(size=n)
    x, t = rng.normal(size=(B, k)), rng.normal(size=(B, n))
    loss, grads = mlp.loss_and_grads([(W, b)], x, t)
    y = np.array([[sum(x[r, c] * W[o, c] for c in range(k)) + b[o] for o in range(n)]
                  for r in range(B)])
    assert loss == pytest.approx(sum((y[r, o] - t[r, o]) ** 2 for r in range(B)
                                     for o in range(n)) / (B * n), rel=1e-14)
    gW = np.array([[sum(2 * (y[r, o] - t[r, o]) * x[r, c] for r in range(B)) / (B * n)
                    for c in range(k)] for o in range(n)])
    gb = np.array([sum(2 * (y[r, o] - t[r, o]) for r in range(B)) / (B * n) for o in range(n)])
    assert np.allclose(grads[0][0], gW, rtol=1e-13, atol=0)
    assert np.allclose(grads[0][1], gb, rtol=1e-13, atol=0)


def test_gradients_match_central_differences():
    """Every weight and bias of a 6 -> 4 x 12 -> 10 net against central differences of the
    loss: relative error <= 1e-6 per tensor."""
    sizes = [6, 12, 12, 12, 12, 10]
    params = _params(sizes, 7)
    rng = np.random.default_rng(8)
    x, t = rng.normal(size=(9, 6)), rng.normal(size=(9, 10))
    _, grads = mlp.loss_and_grads(params, x, t)
    h = 1e-5
    for l in range(len(params)):
        for q in range(2):
            g = grads[l][q]
            fd = np.zeros_like(g)
            for idx in np.ndindex(g.shape):
                for sgn in (1, -1):
                    p2 = [(W.copy(), b.copy()) for W, b in params]
                    p2[l][q][idx] += sgn * h
                    fd[idx] += sgn * mlp.loss_and_grads(p2, x, t)[0]
                fd[idx] /= 2 * h
            assert np.linalg.norm(fd - g) <= 1e-6 * np.linalg.norm(g), (l, q)


def test_adam_first_step_moves_by_lr_times_sign():
    """Bias correction makes the first Adam step exactly -lr g / (|g| + eps)."""
    params = _params([4, 3], 3)
    grads = [(np.array([[1.0, -2.0, 0.5, 3.0]] * 3), np.array([-1.0, 2.0, 0.25]))]
    opt = mlp.Adam(params, lr=0.01, eps=1e-8)
    new = opt.step(params, grads)
    for (W, b), (W1, b1), (gW, gb) in zip(params, new, grads):
        assert np.allclose(W1 - W, -0.01 * gW / (np.abs(gW) + 1e-8), rtol=1e-12, atol=0)
        assert np.allclose(b1 - b, -0.01 * gb / (np.abs(gb) + 1e-8), rtol=1e-12, atol=0)
    # a second identical gradient: m_hat = g and v_hat = g^2 again
    new2 = opt.step(new, grads)
    assert np.allclose(new2[0][0] - new[0][0], -0.01 * grads[0][0] / (np.abs(grads[0][0]) + 1e-8),
                       rtol=1e-9, atol=0)


def test_training_the_oracle_fits_a_smooth_map():
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (256, 6))
    t = np.stack([np.sin(2 * x[:, 0] + x[:, 1]), x[:, 2] * x[:, 3]], axis=1)
    params = _params([6, 32, 32, 2], 9)
    opt = mlp.Adam(params, lr=3e-3)
    first = None
    for it in range(300):
        loss, grads = mlp.loss_and_grads(params, x, t)
        first = loss if first is None else first
        params = opt.step(params, grads)
    assert loss < 0.05 * first
