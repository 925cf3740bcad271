"""FP64 oracle of the proper orthogonal decomposition of solver snapshots (test
infrastructure only: only tests/, the smoke check and the benchmark's CPU arm load it).

The surrogate's outputs are POD coefficients of the solver's displacement fields (the
configuration's "POD coefficients of the peak-systole displacement field"). The plain
definition: with snapshots X [n][D], mean m = column mean, centred X_c = X - m, and the
singular value decomposition X_c = U Sigma W^T (singular values descending), the r modes
are phi = W[:, :r] (orthonormal columns, D x r), the coefficients X_c phi = U Sigma[:, :r],
the eigenvalues lambda_k = sigma_k^2 of X_c X_c^T, and the captured fraction
sum_{k<r} lambda_k / sum_k lambda_k. Each mode is defined up to its sign; the reference
sign makes the mode's largest-magnitude coefficient over the snapshots positive.
"""
from __future__ import annotations

import numpy as np


def pod(X, r: int):
    """(mean [D], phi [D][r], coef [n][r], lam [r], captured fraction) of snapshots X [n][D]."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=0)
    Xc = X - mean[None, :]
    U, sig, Wt = np.linalg.svd(Xc, full_matrices=False)
    phi = Wt[:r].T.copy()
    coef = U[:, :r] * sig[None, :r]
    for k in range(r):                                  # reference sign of each mode
        j = int(np.argmax(np.abs(coef[:, k])))
        if coef[j, k] < 0:
            coef[:, k] = -coef[:, k]
            phi[:, k] = -phi[:, k]
    lam = sig ** 2
    total = lam.sum()
    return mean, phi, coef, lam[:r].copy(), float(lam[:r].sum() / total) if total > 0 else 1.0
