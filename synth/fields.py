"""Nodal Gaussian random fields with Matern covariance on a triangulated surface.

The sampler follows the SPDE route of the paper's Section 2.1 (Eq. 1 and the SPDE
(kappa^2 - Laplacian)^(alpha/2) x = W): with nu = 1 on a 2-D surface, alpha = 2 and the
Galerkin precision is Q = (kappa^2 C~ + G) C~^-1 (kappa^2 C~ + G), where C~ is the lumped
(diagonal) P1 mass matrix and G the P1 stiffness matrix of the surface. A draw with
covariance Q^-1 is x = K^-1 C~^(1/2) z with K = kappa^2 C~ + G and z ~ N(0, I), because
K^-1 C~ K^-1 = Q^-1 (K is symmetric). The paper instead solves with the transposed
Cholesky factor of Q; both give the same distribution.

The continuum marginal variance for nu = 1, d = 2 is 1 / (4 pi kappa^2) (Section 2.1), so
x is multiplied by sigma * sqrt(4 pi) * kappa to give marginal standard deviation sigma.
kappa follows from the correlation length rho = sqrt(8 nu) / kappa.

This is input generation: neither the solver library nor its oracle runs any of it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import kv, gamma


def _philox(seed: int, stream: int, sample: int) -> np.random.Generator:
    """Counter-based generator keyed by (seed, stream, sample): reproducible on any host."""
    key = (int(seed) & 0xFFFFFFFF) | ((int(stream) & 0xFFFF) << 32) | ((int(sample) & 0xFFFF) << 48)
    return np.random.Generator(np.random.Philox(key=key))


def surface_mass_stiffness(xyz: np.ndarray, tri: np.ndarray):
    """Lumped P1 mass C~ (vector) and P1 stiffness G (CSR) of the surface mesh."""
    X = xyz[tri]                                   # [E][3][3]
    e1 = X[:, 1] - X[:, 0]
    e2 = X[:, 2] - X[:, 0]
    n = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(n, axis=1)
    # gradients of the barycentric basis functions on each triangle (in 3-D)
    nh = n / (2.0 * area)[:, None]                 # unit normal
    g = np.empty((tri.shape[0], 3, 3))
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        edge = X[:, c] - X[:, b]                   # edge opposite corner a
        g[:, a] = np.cross(nh, edge) / (2.0 * area)[:, None]
    rows, cols, vals = [], [], []
    for a in range(3):
        for b in range(3):
            rows.append(tri[:, a])
            cols.append(tri[:, b])
            vals.append(area * np.einsum("ij,ij->i", g[:, a], g[:, b]))
    N = xyz.shape[0]
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    Cl = np.zeros(N)
    for a in range(3):
        np.add.at(Cl, tri[:, a], area / 3.0)
    return Cl, G


def gmrf_fields(xyz: np.ndarray, tri: np.ndarray, n_samples: int, corr_length: float,
                std: float, seed: int, streams=(1,), sample0: int = 0) -> list:
    """Zero-mean Matern (nu = 1) fields with marginal std `std`: one [N][S] array per
    entry of `streams` (independent draws sharing one factorisation). Realisation j of the
    result is realisation sample0 + j of the seeded ensemble (its normals are keyed by that
    index), so shards of one ensemble can be drawn apart."""
    N = xyz.shape[0]
    if n_samples == 0:
        return [np.zeros((N, 0)) for _ in streams]
    kappa = np.sqrt(8.0) / corr_length
    Cl, G = surface_mass_stiffness(xyz, tri)
    K = (sp.diags(kappa ** 2 * Cl) + G).tocsc()
    lu = spla.splu(K, permc_spec="COLAMD")
    out = []
    for stream in streams:
        z = np.empty((N, n_samples))
        for s in range(n_samples):
            z[:, s] = _philox(seed, stream, sample0 + s).standard_normal(N)
        x = lu.solve(np.sqrt(Cl)[:, None] * z)
        out.append(x * (std * np.sqrt(4.0 * np.pi) * kappa))
    return out


def lognormal_fields(mesh, n_samples: int, E_mean: float = 0.7e6, h_mean: float = 1.0e-3,
                     corr_length: float = 0.02, std: float = 0.1, seed: int = 0,
                     uniform: bool = False, sample0: int = 0):
    """Nodal E = E_mean exp(g_E), h = h_mean exp(g_h) with independent Matern fields g_E, g_h.

    Returns (E, h), each [N][S] float64 with the sample index innermost.
    uniform=True returns constant fields (g = 0) for closed-form checks.
    """
    N = mesh.n_nodes
    if uniform or std == 0.0:
        return np.full((N, n_samples), E_mean), np.full((N, n_samples), h_mean)
    gE, gh = gmrf_fields(mesh.xyz, mesh.tri, n_samples, corr_length, std, seed, streams=(1, 2),
                         sample0=sample0)
    return E_mean * np.exp(gE), h_mean * np.exp(gh)


def gaussian_fields(mesh, n_samples: int, E_mean: float, E_std: float, h_mean: float, h_std: float,
                    corr_length: float, seed: int = 0):
    """Nodal E = E_mean + g_E, h = h_mean + g_h with independent Matern fields of marginal
    standard deviations E_std and h_std (the Gaussian marginals of the paper's cylinder
    benchmark). Returns (E, h), each [N][S] float64."""
    gE, gh = gmrf_fields(mesh.xyz, mesh.tri, n_samples, corr_length, 1.0, seed, streams=(1, 2))
    return E_mean + E_std * gE, h_mean + h_std * gh


def matern_correlation(d, corr_length: float, nu: float = 1.0):
    """Matern correlation r(d)/sigma^2 = 2^(1-nu)/Gamma(nu) (kappa d)^nu K_nu(kappa d), Eq. 1."""
    d = np.asarray(d, dtype=np.float64)
    kappa = np.sqrt(8.0 * nu) / corr_length
    kd = kappa * d
    out = np.ones_like(kd)
    nz = kd > 0
    out[nz] = (2.0 ** (1.0 - nu) / gamma(nu)) * kd[nz] ** nu * kv(nu, kd[nz])
    return out
