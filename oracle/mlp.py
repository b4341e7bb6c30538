"""FP64 MLP oracle for the S-parameter surrogate.

TEST INFRASTRUCTURE ONLY (tests/, bench.py's CPU legs).  Shares no code with the CUDA
library; the surrogate is not in the paper (which characterises each line by a full FDTD run,
Sec. II-A); the network follows the surrogate workload's own statement:

  6 line descriptors -> 4 hidden layers of 512 with GELU -> 512 outputs
  (Re/Im of S11 and S21 at 128 frequencies), mean-squared-error loss, Adam.

Conventions (the same ones the GPU kernels implement):
  * layer l: z_l = a_{l-1} W_l^T + b_l, W_l of shape (out, in), rows of a are samples;
    a_l = gelu(z_l) for the hidden layers, the last layer is linear;
  * gelu in its tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (Hendrycks and
    Gimpel's approximation; the GPU evaluates the same expression);
  * loss = mean over all batch x output entries of (y - t)^2;
  * Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps) at step k = 1, 2, ...
Plain numpy in float64, one matrix product per layer and direction, no fusion.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

C_GELU = math.sqrt(2.0 / math.pi)
A_GELU = 0.044715

Params = List[Tuple[np.ndarray, np.ndarray]]


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + A_GELU * x ** 3)))


def gelu_grad(x: np.ndarray) -> np.ndarray:
    """d gelu / dx of the tanh form."""
    th = np.tanh(C_GELU * (x + A_GELU * x ** 3))
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * C_GELU * (1.0 + 3.0 * A_GELU * x * x)


def forward(params: Params, x: np.ndarray):
    """Returns (y, cache); cache = (activations a_0..a_{L-1}, pre-activations z_1..z_L)."""
    a = [np.asarray(x, dtype=np.float64)]
    z = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        zl = a[-1] @ W.T + b
        z.append(zl)
        if l < L - 1:
            a.append(gelu(zl))
    return z[-1], (a, z)


def mse(y: np.ndarray, t: np.ndarray) -> float:
    return float(np.mean((y - t) ** 2))


def mse_grad(y: np.ndarray, t: np.ndarray) -> np.ndarray:
    return 2.0 * (y - t) / y.size


def backward(params: Params, cache, dy: np.ndarray) -> Params:
    """Gradients (dW_l, db_l) of a scalar whose gradient with respect to y is dy."""
    a, z = cache
    L = len(params)
    grads: Params = [None] * L
    dz = dy
    for l in range(L - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (dz.T @ a[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * gelu_grad(z[l - 1])
    return grads


def loss_and_grads(params: Params, x: np.ndarray, t: np.ndarray):
    y, cache = forward(params, x)
    return mse(y, t), backward(params, cache, mse_grad(y, t))


class Adam:
    def __init__(self, params: Params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.k = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params: Params, grads: Params) -> Params:
        self.k += 1
        c1 = 1.0 - self.b1 ** self.k
        c2 = 1.0 - self.b2 ** self.k
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for q, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][q] + (1.0 - self.b1) * g
                v = self.b2 * self.v[l][q] + (1.0 - self.b2) * g * g
                self.m[l] = self.m[l][:q] + (m,) + self.m[l][q + 1:]
                self.v[l] = self.v[l][:q] + (v,) + self.v[l][q + 1:]
                new.append(p - self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            out.append((new[0], new[1]))
        return out
