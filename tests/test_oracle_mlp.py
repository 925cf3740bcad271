"""Pins of the surrogate-network oracle.

* Gradients against central finite differences of the loss (every parameter tensor).
* GELU against its special values and symmetry: g(0) = 0, g(z) - g(-z) = z, g' from a
  finite difference.
* Adam's first step moves every parameter by lr * g / (|g| + eps / ...) which, with the
  bias corrections, is lr * sign(g) up to eps: a closed form independent of the code path.
* Adam's later steps against the unrolled form of its recurrences: the bias-corrected
  moments are normalised exponentially weighted means of the gradient history.
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


def test_forward_reduces_to_the_affine_map_when_gelu_is_linear():
    """With every pre-activation far above zero, GELU(z) = z up to z * Phi(-z) < 1e-20, so
    the network is the product of its affine maps (a closed form of the layer order and
    the (out, in) weight convention)."""
    rng = np.random.default_rng(5)
    sizes = [4, 6, 5, 3]
    W1 = rng.uniform(0.5, 1.0, (6, 4))
    W2 = rng.uniform(0.5, 1.0, (5, 6))
    W3 = rng.standard_normal((3, 5))
    b1, b2, b3 = np.full(6, 20.0), np.full(5, 20.0), rng.standard_normal(3)
    x = rng.uniform(0.0, 1.0, (7, 4))
    y, _ = mlp.forward([W1, b1, W2, b2, W3, b3], x)
    ref = ((x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(y, ref, rtol=1e-13, atol=0)


def test_hidden_unit_permutation_and_loss_definition():
    rng = np.random.default_rng(6)
    params = mlp.init_params([5, 8, 8, 2], seed=4)
    x = rng.standard_normal((9, 5))
    y, _ = mlp.forward(params, x)
    p1, p2 = rng.permutation(8), rng.permutation(8)
    W1, b1, W2, b2, W3, b3 = params
    perm = [W1[p1], b1[p1], W2[p2][:, p1], b2[p2], W3[:, p2], b3]
    assert np.allclose(mlp.forward(perm, x)[0], y, rtol=1e-14, atol=1e-15)
    t = y + 0.5                       # every residual is -0.5
    assert mlp.loss(params, x, t) == pytest.approx(0.25, rel=1e-14)


def test_adam_later_steps_match_the_weighted_mean_closed_form():
    """Adam beyond its first step. Unrolling m_t = b1 m_{t-1} + (1 - b1) g_t from m_0 = 0
    gives m_t = (1 - b1) sum_k b1^(t-k) g_k, and 1 - b1^t = (1 - b1) sum_{j<t} b1^j, so the
    bias-corrected moment is the normalised exponentially weighted mean
        mhat_t = sum_k b1^(t-k) g_k / sum_k b1^(t-k)
    (likewise vhat_t with b2 and g_k^2). The parameter after T steps is therefore
    p_0 - lr sum_t mhat_t / (sqrt(vhat_t) + eps), written here from those weighted means
    over the whole gradient history, not from the recurrence. Distinct gradients per step
    and b1 != b2 make a swapped beta, a wrong bias-correction exponent or a moment that is
    not carried between steps fail."""
    rng = np.random.default_rng(11)
    shape = (4, 5)
    T = 5
    gs = [rng.standard_normal(shape) * (1.0 + 0.5 * t) for t in range(T)]
    p0 = rng.standard_normal(shape)
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    params = [p0.copy()]
    opt = mlp.Adam(params, lr=lr, b1=b1, b2=b2, eps=eps)
    expect = p0.copy()
    for t in range(1, T + 1):
        opt.step(params, [gs[t - 1]])
        w1 = np.array([b1 ** (t - k) for k in range(1, t + 1)])
        w2 = np.array([b2 ** (t - k) for k in range(1, t + 1)])
        hist = np.stack(gs[:t])
        mhat = np.tensordot(w1, hist, axes=1) / w1.sum()
        vhat = np.tensordot(w2, hist * hist, axes=1) / w2.sum()
        expect = expect - lr * mhat / (np.sqrt(vhat) + eps)
        assert np.allclose(params[0], expect, rtol=1e-12, atol=1e-14), t
    # the closed form itself is not symmetric in (b1, b2): swapping them moves step 2
    q = [p0.copy()]
    swapped = mlp.Adam(q, lr=lr, b1=b2, b2=b1, eps=eps)
    for t in range(2):
        swapped.step(q, [gs[t]])
    p2 = [p0.copy()]
    right = mlp.Adam(p2, lr=lr, b1=b1, b2=b2, eps=eps)
    for t in range(2):
        right.step(p2, [gs[t]])
    assert np.abs(q[0] - p2[0]).max() > 1e-4
