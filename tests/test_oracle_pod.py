"""Pins of the POD oracle (oracle/pod.py).

* Snapshots built from known orthonormal modes W, orthogonal coefficient columns and
  singular values s (X = m + U diag(s) W^T with U^T U = I and columns of U summing to zero,
  so that the column mean is m) give back m, s^2 as the eigenvalues, the modes and
  coefficients up to sign, and the captured fraction sum_{k<r} s_k^2 / sum s^2.
* Eckart-Young: the rank-r reconstruction error ||X_c - coef phi^T||_F^2 equals the sum of
  the discarded eigenvalues, and no other rank-r projection (here random ones) does better.
* The modes are orthonormal and the coefficients are the projections X_c phi.
"""
import numpy as np
import pytest

from oracle import pod as op


def _known(n=40, D=300, q=6, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, q))
    A -= A.mean(axis=0)                       # columns sum to zero: the mean is m
    U, _ = np.linalg.qr(A)
    W, _ = np.linalg.qr(rng.standard_normal((D, q)))
    s = np.array([9.0, 5.0, 3.0, 1.5, 0.7, 0.2])[:q]
    m = rng.standard_normal(D)
    return m[None, :] + (U * s[None, :]) @ W.T, m, U, W, s


def test_known_modes_and_singular_values():
    X, m, U, W, s = _known()
    mean, phi, coef, lam, frac = op.pod(X, 4)
    assert np.allclose(mean, m, atol=1e-12)
    assert np.allclose(lam, s[:4] ** 2, rtol=1e-12)
    assert frac == pytest.approx((s[:4] ** 2).sum() / (s ** 2).sum(), rel=1e-12)
    for k in range(4):
        sgn = np.sign(phi[:, k] @ W[:, k])
        assert np.allclose(sgn * phi[:, k], W[:, k], atol=1e-10)
        assert np.allclose(sgn * coef[:, k], U[:, k] * s[k], atol=1e-10)
        j = np.argmax(np.abs(coef[:, k]))
        assert coef[j, k] > 0                 # the reference sign


def test_eckart_young_and_orthonormality():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30, 120)) @ np.diag(np.linspace(3, 0.1, 120))
    r = 7
    mean, phi, coef, lam, _ = op.pod(X, r)
    Xc = X - mean
    assert np.allclose(phi.T @ phi, np.eye(r), atol=1e-12)
    assert np.allclose(coef, Xc @ phi, atol=1e-10)
    err = np.linalg.norm(Xc - coef @ phi.T) ** 2
    lam_all = np.linalg.svd(Xc, compute_uv=False) ** 2
    assert err == pytest.approx(lam_all[r:].sum(), rel=1e-10)
    for _ in range(5):
        Q, _ = np.linalg.qr(rng.standard_normal((120, r)))
        assert np.linalg.norm(Xc - (Xc @ Q) @ Q.T) ** 2 > err
