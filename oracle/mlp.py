"""FP64 CPU oracle of the surrogate network (test infrastructure only).

A multilayer perceptron x -> GELU(x W1^T + b1) -> GELU(. W2^T + b2) -> . W3^T + b3 with
the exact GELU g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2, a mean-squared-error loss
L = sum((y - t)^2) / (B * n_out), reverse-mode gradients written out layer by layer, and
the Adam update (Kingma & Ba 2015: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
theta <- theta - lr * mhat / (sqrt(vhat) + eps) with bias-corrected mhat, vhat). Used to
check the device kernels' forward pass, gradients and optimiser. Weights follow the
(out, in) convention of y = x W^T + b.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def init_params(sizes, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (float64)."""
    rng = np.random.default_rng(seed)
    params = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        bound = 1.0 / np.sqrt(fi)
        params.append(rng.uniform(-bound, bound, size=(fo, fi)))
        params.append(rng.uniform(-bound, bound, size=(fo,)))
    return params


def forward(params, x):
    """Returns (y, cache) with cache = pre-activations and activations per layer."""
    a = np.asarray(x, dtype=np.float64)
    acts, pres = [a], []
    n_layers = len(params) // 2
    for l in range(n_layers):
        W, b = params[2 * l], params[2 * l + 1]
        z = a @ W.T + b
        pres.append(z)
        a = gelu(z) if l < n_layers - 1 else z
        acts.append(a)
    return a, (acts, pres)


def loss(params, x, t):
    y, _ = forward(params, x)
    d = y - t
    return float(np.sum(d * d) / d.size)


def gradients(params, x, t):
    """Loss and dL/dparams by reverse-mode differentiation of the layers above."""
    y, (acts, pres) = forward(params, x)
    n_layers = len(params) // 2
    d = y - t
    L = float(np.sum(d * d) / d.size)
    g = 2.0 * d / d.size                     # dL/dy
    grads = [None] * len(params)
    for l in reversed(range(n_layers)):
        if l < n_layers - 1:
            g = g * gelu_grad(pres[l])       # through the activation
        grads[2 * l] = g.T @ acts[l]         # dL/dW = g^T a_prev
        grads[2 * l + 1] = g.sum(axis=0)     # dL/db
        g = g @ params[2 * l]                # dL/da_prev
    return L, grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            mhat = m / (1.0 - self.b1 ** self.t)
            vhat = v / (1.0 - self.b2 ** self.t)
            p -= self.lr * mhat / (np.sqrt(vhat) + self.eps)
