"""Truncated Karhunen-Loeve parametrisation of the random wall fields (input generation).

The covariance is the one the SPDE/GMRF sampler draws from (synth.fields): with
K = kappa^2 C~ + G and the variance scale s = sigma sqrt(4 pi) kappa, a draw is
x = s K^-1 C~^(1/2) z, so Cov(x) = s^2 K^-1 C~ K^-1. Its leading eigenpairs (lambda_k, v_k)
give the truncated expansion g = sum_k sqrt(lambda_k) xi_k v_k with xi_k ~ N(0, 1), which is
how the surrogate's inputs (32 coefficients for E, 32 for h) define a realisation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fields import surface_mass_stiffness, _philox


def kl_basis(mesh, n_modes: int = 32, corr_length: float = 0.02, std: float = 0.1):
    """(lambda [n_modes] descending, V [N][n_modes] orthonormal) of the field covariance."""
    kappa = np.sqrt(8.0) / corr_length
    Cl, G = surface_mass_stiffness(mesh.xyz, mesh.tri)
    K = (sp.diags(kappa ** 2 * Cl) + G).tocsc()
    lu = spla.splu(K, permc_spec="COLAMD")
    s2 = (std * np.sqrt(4.0 * np.pi) * kappa) ** 2
    N = mesh.n_nodes
    op = spla.LinearOperator((N, N), matvec=lambda v: s2 * lu.solve(Cl * lu.solve(np.ravel(v))),
                             dtype=np.float64)
    lam, V = spla.eigsh(op, k=n_modes, which="LA", tol=1e-8)
    order = np.argsort(-lam)
    return lam[order], np.ascontiguousarray(V[:, order])


def kl_coefficients(n: int, n_modes: int, seed: int, first: int = 0) -> np.ndarray:
    """xi [n][2 n_modes] ~ N(0, 1) (E coefficients then h coefficients), row i seeded by (seed, first + i)."""
    out = np.empty((n, 2 * n_modes))
    for i in range(n):
        out[i] = _philox(seed, 7, first + i).standard_normal(2 * n_modes)
    return out


def kl_fields(basis, xi: np.ndarray, E_mean: float = 0.7e6, h_mean: float = 1.0e-3):
    """Nodal E, h [N][S] for coefficient rows xi [S][2 n_modes]."""
    lam, V = basis
    n = lam.shape[0]
    sq = np.sqrt(lam)
    gE = V @ (xi[:, :n] * sq[None, :]).T
    gh = V @ (xi[:, n:2 * n] * sq[None, :]).T
    return np.ascontiguousarray(E_mean * np.exp(gE)), np.ascontiguousarray(h_mean * np.exp(gh))
