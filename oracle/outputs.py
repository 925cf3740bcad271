"""FP64 oracle of the ensemble output statistics. Test infrastructure only: only tests/,
the smoke check and the benchmark's CPU arm load it.

Section 3 reports, over the realisations of one ensemble, mean displacement magnitudes
with 5 %-95 % bands, time histories of displacement and stress at chosen locations, and
stress components in a local cylindrical frame (Section 2.2.3: axial = tangent of the
closest centreline location, radial = the wall normal at the point, circumferential =
their cross product). The stress is the solid stress of Section 2.2.1, sigma = C B u in
the element frame with the printed B and C.

Readings (the paper names the quantities but not these details):
  * quantiles are of type 7 (Hyndman and Fan): sorted x_0..x_{S-1}, h = p (S - 1),
    Q(p) = x_j + (h - j)(x_{j+1} - x_j), j = floor(h);
  * E in C is the element mean of the nodal modulus (the average of the linear field
    over the three Gauss points), one stress per element;
  * the stress is evaluated at the element centroid with the frame there; the axial
    direction is the centreline tangent projected on the wall (so the frame is
    orthonormal), theta = r x t normalised, r the outward normal (X2 - X1) x (X3 - X1);
  * the variance divisor is S - 1.
"""
from __future__ import annotations

import numpy as np


def quantiles(rows: np.ndarray, q) -> np.ndarray:
    """Type-7 quantiles of every row of rows [n][S] at probabilities q: [n][len(q)]."""
    x = np.sort(np.asarray(rows, dtype=np.float64), axis=1)
    S = x.shape[1]
    out = np.empty((x.shape[0], len(q)))
    for k, p in enumerate(q):
        h = float(p) * (S - 1)
        j = min(int(np.floor(h)), S - 1)
        j1 = min(j + 1, S - 1)
        g = h - j
        out[:, k] = x[:, j] + g * (x[:, j1] - x[:, j])
    return out


def row_stats(rows: np.ndarray, q=()):
    """(mean, sample variance with divisor S - 1, quantiles) of every row."""
    rows = np.asarray(rows, dtype=np.float64)
    S = rows.shape[1]
    mean = rows.sum(axis=1) / S
    var = ((rows - mean[:, None]) ** 2).sum(axis=1) / (S - 1) if S > 1 else np.zeros(rows.shape[0])
    return mean, var, (quantiles(rows, q) if len(q) else None)


def displacement_rows(u_snc: np.ndarray) -> np.ndarray:
    """Rows (node, dof) [N * 3][S] of displacements given as [S][N][3]."""
    S = u_snc.shape[0]
    return np.ascontiguousarray(np.transpose(u_snc, (1, 2, 0)).reshape(-1, S))


def magnitude_rows(u_snc: np.ndarray) -> np.ndarray:
    """|u| per node and realisation: [N][S]."""
    return np.ascontiguousarray(np.linalg.norm(u_snc, axis=2).T)


def peak_magnitude(model, n_steps: int, stride: int = 1, up=None, uc=None, step0: int = 0, peak=None):
    """Running peak of the displacement magnitude (Section 3's peak and band quantities
    over a heart cycle): for every node and realisation, the largest |u_k| over the
    recorded steps k, the multiples of `stride` in (step0, step0 + n_steps]. Starts from
    rest unless (up, uc) = (u_{step0 - 1}, u_{step0}) [S][N][3] and a previous peak [N][S]
    are given. Returns (peak [N][S], u_prev, u_cur) after the last step; steps with
    model.steps, one recording interval at a time."""
    if up is None:
        up, uc = model.start()
    peak = np.zeros((model.N, model.S)) if peak is None else np.array(peak, dtype=np.float64)
    step, end = step0, step0 + n_steps
    while step < end:
        k = min(stride - step % stride, end - step)
        model.steps(up, uc, step, k)
        step += k
        if step % stride == 0:
            peak = np.maximum(peak, magnitude_rows(uc))
    return peak, up, uc


def _frames(xyz, tri):
    X = xyz[tri]
    d12 = X[:, 1] - X[:, 0]
    d13 = X[:, 2] - X[:, 0]
    n = np.cross(d12, d13)
    A2 = np.linalg.norm(n, axis=1)
    n = n / A2[:, None]
    e1 = d12 / np.linalg.norm(d12, axis=1)[:, None]   # edge 1 -> 2
    e2 = np.cross(n, e1)
    return X, e1, e2, n, A2


def _closest_tangent(c: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Unit tangent of the centreline segment closest to each point of c (first on ties)."""
    P0, P1 = pts[:-1], pts[1:]
    d = P1 - P0
    dd = np.einsum("ij,ij->i", d, d)
    best = np.full(c.shape[0], np.inf)
    t = np.zeros_like(c)
    for k in range(d.shape[0]):
        if dd[k] <= 0:
            continue
        w = c - P0[k]
        tau = np.clip(w @ d[k] / dd[k], 0.0, 1.0)
        r = w - tau[:, None] * d[k]
        dist = np.einsum("ij,ij->i", r, r)
        upd = dist < best
        best[upd] = dist[upd]
        t[upd] = d[k] / np.sqrt(dd[k])
    return t


def element_stress(xyz, tri, u_snc, E_node, nu, kshear, centerline) -> np.ndarray:
    """Stress rows (element, k) [E * 6][S], k = rr, tt, zz, rt, rz, tz."""
    xyz = np.asarray(xyz, dtype=np.float64)
    X, e1, e2, n, A2 = _frames(xyz, tri)
    E = tri.shape[0]
    S = u_snc.shape[0]
    # local coordinates
    x = np.stack([np.einsum("ij,ij->i", X[:, a] - X[:, 0], e1) for a in range(3)], axis=1)
    y = np.stack([np.einsum("ij,ij->i", X[:, a] - X[:, 0], e2) for a in range(3)], axis=1)
    y23, y31, y12 = y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]
    x32, x13, x21 = x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]
    B = np.zeros((E, 5, 9))
    for a, (ya, xa) in enumerate(((y23, x32), (y31, x13), (y12, x21))):
        B[:, 0, 3 * a] = ya
        B[:, 1, 3 * a + 1] = xa
        B[:, 2, 3 * a] = xa
        B[:, 2, 3 * a + 1] = ya
        B[:, 3, 3 * a + 2] = ya
        B[:, 4, 3 * a + 2] = xa
    B /= A2[:, None, None]
    C0 = np.array([[1, nu, 0, 0, 0], [nu, 1, 0, 0, 0], [0, 0, 0.5 * (1 - nu), 0, 0],
                   [0, 0, 0, 0.5 * kshear * (1 - nu), 0], [0, 0, 0, 0, 0.5 * kshear * (1 - nu)]]) / (1 - nu * nu)
    Lam = np.stack([e1, e2, n], axis=1)                   # [E][3][3], rows e1, e2, n
    # cylindrical frame at the centroid
    c = X.mean(axis=1)
    t = _closest_tangent(c, np.asarray(centerline, dtype=np.float64))
    r = n
    th = np.cross(r, t)
    th /= np.linalg.norm(th, axis=1)[:, None]
    z = t - np.einsum("ij,ij->i", t, r)[:, None] * r
    z /= np.linalg.norm(z, axis=1)[:, None]
    R = np.stack([r, th, z], axis=1)                      # [E][3][3], rows r, t, z
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    Ebar = E_node[tri].mean(axis=1)                       # [E][S]
    out = np.empty((E, 6, S))
    for s in range(S):
        ue = u_snc[s][tri]                                # [E][3 nodes][3]
        ul = np.einsum("eij,eaj->eai", Lam, ue).reshape(E, 9)
        eps = np.einsum("eij,ej->ei", B, ul)
        sl = (eps @ C0.T) * Ebar[:, s][:, None]           # sxx, syy, txy, txz, tyz
        T = np.zeros((E, 3, 3))
        T[:, 0, 0], T[:, 1, 1] = sl[:, 0], sl[:, 1]
        T[:, 0, 1] = T[:, 1, 0] = sl[:, 2]
        T[:, 0, 2] = T[:, 2, 0] = sl[:, 3]
        T[:, 1, 2] = T[:, 2, 1] = sl[:, 4]
        G = np.einsum("eji,ejk,ekl->eil", Lam, T, Lam)    # Lambda^T T Lambda (global)
        Cy = np.einsum("eai,eij,ebj->eab", R, G, R)
        for k, (a, b) in enumerate(pairs):
            out[:, k, s] = Cy[:, a, b]
    return out.reshape(E * 6, S)
