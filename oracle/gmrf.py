"""FP64 oracle of the Matérn random-field sampler (Section 2.1). Test infrastructure only:
only tests/, the smoke check and the benchmark's CPU arm load it.

Section 2.1 discretises the SPDE (kappa^2 - Laplacian)^(alpha/2) x = W with piecewise
linear basis functions psi_k on the triangulated surface:

    G_ij = <grad psi_i, grad psi_j>,   C_ij = <psi_i, psi_j>,   C~ = lumped (diagonal) C,

and for alpha = 2 (nu = 1 on a 2-D surface) the precision of the nodal weights is
Q_2 = (kappa^2 C~ + G)^T C~^-1 (kappa^2 C~ + G). Section 2.1 also gives the marginal
variance of the continuous field, Gamma(nu) / (Gamma(nu + d/2) (4 pi)^(d/2) kappa^(2 nu)),
which is 1 / (4 pi kappa^2) here, and relates kappa to the correlation length rho by
rho = sqrt(8 nu) / kappa.

A draw with covariance Q_2^-1 is x = K^-1 C~^(1/2) z with K = kappa^2 C~ + G and
z ~ N(0, I): its covariance is K^-1 C~ K^-1 = Q_2^-1 because K is symmetric. The paper
draws the same distribution through the Cholesky factor of Q_2 (x = L^-T z); the device
sampler uses the two-stage form because it needs only solves with the sparse K, so this
oracle computes the same map from the same z: one sparse direct solve per sample (scipy's
LU as the library step), then the scale sigma sqrt(4 pi) kappa that gives marginal
standard deviation sigma.

Here G is assembled edge by edge with the cotangent formula (G_ij = -(cot a_ij + cot b_ij)/2
for the angles opposite edge ij, G_ii = -sum_j G_ij), and C_ij = A_e (1 + delta_ij) / 12 per
element, lumped by row sums.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def consistent_mass(xyz: np.ndarray, tri: np.ndarray) -> sp.csr_matrix:
    """C_ij = <psi_i, psi_j>: A_e / 6 on the diagonal and A_e / 12 off it, per element."""
    X = xyz[tri]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tri[:, a])
            cols.append(tri[:, b])
            vals.append(area * (2.0 if a == b else 1.0) / 12.0)
    N = xyz.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def lumped_mass(xyz: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """C~_ii = sum_j C_ij (row sums of the consistent mass)."""
    return np.asarray(consistent_mass(xyz, tri).sum(axis=1)).ravel()


def stiffness(xyz: np.ndarray, tri: np.ndarray) -> sp.csr_matrix:
    """G_ij = <grad psi_i, grad psi_j> by the cotangent formula."""
    rows, cols, vals = [], [], []
    for a in range(3):
        i, j, k = tri[:, a], tri[:, (a + 1) % 3], tri[:, (a + 2) % 3]
        # angle at corner k, opposite edge (i, j)
        u = xyz[i] - xyz[k]
        v = xyz[j] - xyz[k]
        cot = np.einsum("ij,ij->i", u, v) / np.linalg.norm(np.cross(u, v), axis=1)
        w = -0.5 * cot
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [w, w, -w, -w]
    N = xyz.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def operator(xyz: np.ndarray, tri: np.ndarray, kappa: float):
    """(K = kappa^2 C~ + G, C~)."""
    Cl = lumped_mass(xyz, tri)
    return (sp.diags(kappa * kappa * Cl) + stiffness(xyz, tri)).tocsc(), Cl


def precision(xyz: np.ndarray, tri: np.ndarray, kappa: float) -> sp.csr_matrix:
    """Q_2 = K^T C~^-1 K exactly as Section 2.1 writes it for alpha = 2."""
    K, Cl = operator(xyz, tri, kappa)
    return (K.T @ sp.diags(1.0 / Cl) @ K).tocsr()


def kappa_of(corr_length: float, nu: float = 1.0) -> float:
    """kappa = sqrt(8 nu) / rho (Section 2.1)."""
    return np.sqrt(8.0 * nu) / corr_length


def marginal_scale(kappa: float, sigma: float) -> float:
    """Factor taking the nu = 1, d = 2 solution (variance 1 / (4 pi kappa^2)) to marginal
    standard deviation sigma."""
    return sigma * np.sqrt(4.0 * np.pi) * kappa


def sample(xyz: np.ndarray, tri: np.ndarray, kappa: float, z: np.ndarray) -> np.ndarray:
    """x = K^-1 C~^(1/2) z for every column of z ([N][S], sample index innermost)."""
    K, Cl = operator(xyz, tri, kappa)
    lu = spla.splu(K, permc_spec="COLAMD")
    return lu.solve(np.sqrt(Cl)[:, None] * np.asarray(z, dtype=np.float64))
