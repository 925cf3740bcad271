"""Pins of the surrogate-network oracle.

* Gradients against central finite differences of the loss (every parameter tensor).
* GELU against its special values and symmetry: g(0) = 0, g(z) - g(-z) = z, g' from a
  finite difference.
* Adam's first step moves every parameter by lr * g / (|g| + eps / ...) which, with the
  bias corrections, is lr * sign(g) up to eps: a closed form independent of the code path.
"""
import numpy as np
import pytest

from oracle import mlp


def test_gelu_identities():
    z = np.linspace(-6, 6, 101)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    sizes = [6, 9, 7, 4]
    params = mlp.init_params(sizes, seed=1)
    x = rng.standard_normal((5, 6))
    t = rng.standard_normal((5, 4))
    L, grads = mlp.gradients(params, x, t)
    assert L == pytest.approx(mlp.loss(params, x, t), rel=1e-15)
    h = 1e-6
    for p, g in zip(params, grads):
        fd = np.zeros_like(p)
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[idx]
            p[idx] = old + h
            lp = mlp.loss(params, x, t)
            p[idx] = old - h
            lm = mlp.loss(params, x, t)
            p[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(0)
    params = [rng.standard_normal((3, 4))]
    grads = [rng.standard_normal((3, 4))]
    before = params[0].copy()
    opt = mlp.Adam(params, lr=0.01, eps=1e-12)
    opt.step(params, grads)
    assert np.allclose(params[0] - before, -0.01 * np.sign(grads[0]), rtol=1e-9, atol=0)
