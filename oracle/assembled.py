"""Assembled form of the ensemble stiffness (test infrastructure only).

The paper's CPU solver stores the ensemble stiffness as a CSR matrix whose entries are
3 x 3 node blocks carrying one value per realisation (Section 2.3, entries of size
9 n_s). This module assembles that matrix from the oracle's element matrices, one
scipy CSR matrix per realisation with the same sparsity, so tests can check the
assembly-free product, compute static solutions and generalised eigenvalues.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble(model, sample: int) -> sp.csr_matrix:
    """K_s (3N x 3N) of one realisation: sum_e (E h)_e,s P_e^T Kg_e P_e."""
    tri = model.tri
    E = tri.shape[0]
    dof = (3 * tri[:, :, None] + np.arange(3)[None, None, :]).reshape(E, 9)
    rows = np.repeat(dof, 9, axis=1).ravel()
    cols = np.tile(dof, (1, 9)).ravel()
    vals = (model.Kg.reshape(E, 81) * model.eh_se[sample][:, None]).ravel()
    n = 3 * model.N
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def block_csr(model):
    """Ensemble CSR with 3 x 3 x S blocks: (row_ptr [N+1], col [nnz], blocks [nnz][3][3][S])."""
    tri = model.tri
    N, S = model.N, model.S
    pairs = {}
    for e in range(tri.shape[0]):
        for a in range(3):
            for b in range(3):
                key = (int(tri[e, a]), int(tri[e, b]))
                pairs.setdefault(key, []).append((e, a, b))
    keys = sorted(pairs)
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    for (i, _j) in keys:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    col = np.array([j for (_i, j) in keys], dtype=np.int64)
    Kg = model.Kg.reshape(-1, 9, 9)
    blocks = np.zeros((len(keys), 3, 3, S))
    for k, key in enumerate(keys):
        for (e, a, b) in pairs[key]:
            blk = Kg[e, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
            blocks[k] += blk[:, :, None] * model.eh_se[:, e][None, None, :]
    return row_ptr, col, blocks


def block_csr_matvec(row_ptr, col, blocks, u_n3s):
    """y[i][:, s] = sum_k blocks[k][:, :, s] u[col[k]][:, s] for the block CSR above."""
    N = row_ptr.shape[0] - 1
    y = np.zeros_like(u_n3s)
    for i in range(N):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            y[i] += np.einsum("abs,bs->as", blocks[k], u_n3s[col[k]])
    return y


def lumped_mass_vector(model, sample: int) -> np.ndarray:
    """Diagonal of M~ for one realisation, repeated over the 3 dofs of each node."""
    return np.repeat(model.m_sn[sample], 3)
