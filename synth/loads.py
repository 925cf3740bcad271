"""Wall traction histories (inputs only).

The paper's structural solver receives, at every wall node, the three components of
the nodal force built from the fluid wall stress (Section 2.2.3: shear and normals of
adjacent elements are averaged and the nodal pressure added). With no fluid solver in
scope, loads are synthesised in the separable form f_n = sum_j amp[n][j] * P_j: a few
fixed nodal force patterns P_j ([J][N][3]) times an amplitude table ([n_steps][J]).
A pattern distributes a unit element traction to the element's corners in equal
thirds; pressure acts along the outward element normal (t^s = -t^f with t^f = -p n).
"""
from __future__ import annotations

import numpy as np


def _element_frames(xyz, tri):
    X = xyz[tri]
    n = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    area = 0.5 * np.linalg.norm(n, axis=1)
    n = n / (2.0 * area)[:, None]
    return X, n, area


def pressure_shear_modes(mesh, pressure_weight=None, shear_dir=(0.0, 0.0, 1.0),
                         with_shear: bool = False, delay_modes=None) -> np.ndarray:
    """Nodal force patterns for unit pressure (and optionally unit axial shear).

    pressure_weight: optional per-element multiplier of the unit pressure (e.g. a
    spatial profile); shear_dir: direction whose in-plane projection carries the shear.
    delay_modes: optional [M][E] per-element weights producing extra pressure patterns
    (used for travelling-wave loads, which split into cos/sin spatial patterns).
    Returns [J][N][3] float64.
    """
    X, n, area = _element_frames(mesh.xyz, mesh.tri)
    E = mesh.n_elems
    N = mesh.n_nodes
    weights = [np.ones(E) if pressure_weight is None else np.asarray(pressure_weight, dtype=np.float64)]
    if delay_modes is not None:
        weights = [np.asarray(w, dtype=np.float64) for w in delay_modes]
    modes = []
    for w in weights:
        fe = (area * w / 3.0)[:, None] * n
        P = np.zeros((N, 3))
        for a in range(3):
            np.add.at(P, mesh.tri[:, a], fe)
        modes.append(P)
    if with_shear:
        d = np.asarray(shear_dir, dtype=np.float64)
        t = d[None, :] - np.einsum("ij,j->i", n, d)[:, None] * n
        tn = np.linalg.norm(t, axis=1)
        t = np.where(tn[:, None] > 1e-12, t / np.maximum(tn, 1e-300)[:, None], 0.0)
        fe = (area / 3.0)[:, None] * t
        P = np.zeros((N, 3))
        for a in range(3):
            np.add.at(P, mesh.tri[:, a], fe)
        modes.append(P)
    return np.ascontiguousarray(np.stack(modes))


def step_amplitudes(n_steps: int, value: float, J: int = 1) -> np.ndarray:
    """Constant amplitude `value` on the first pattern from step 0 (a step load)."""
    amp = np.zeros((n_steps, J))
    amp[:, 0] = value
    return amp


def waveform(t, mean: float = 10.7e3, half_range: float = 2.7e3, period: float = 0.8,
             harmonics: int = 5):
    """Pulsatile pressure: 5 cosine harmonics with amplitudes 1/k, zero phase, rescaled
    so that its minimum and maximum over a period are mean -/+ half_range."""
    t = np.asarray(t, dtype=np.float64)
    k = np.arange(1, harmonics + 1)

    def raw(tt):
        return np.sum(np.cos(2 * np.pi * k[None, :] * tt[..., None] / period) / k[None, :], axis=-1)

    grid = np.linspace(0.0, period, 200001)
    w = raw(grid)
    lo, hi = w.min(), w.max()
    return mean + half_range * (2.0 * raw(t) - (hi + lo)) / (hi - lo)


def ramp(t, duration: float = 0.2):
    """Quarter-sine load ramp: sin(pi t / (2 duration)) for t < duration, then 1."""
    t = np.asarray(t, dtype=np.float64)
    return np.where(t < duration, np.sin(0.5 * np.pi * t / duration), 1.0)


def pulsatile_amplitudes(n_steps: int, dt: float, with_shear: bool = True,
                         shear: float = 1.0, ramp_duration: float = 0.2,
                         t0: float = 0.0) -> np.ndarray:
    """Amplitude table [n_steps][J] for (pressure waveform, axial shear) under the ramp."""
    t = t0 + dt * np.arange(n_steps)
    r = ramp(t, ramp_duration)
    cols = [r * waveform(t)]
    if with_shear:
        cols.append(r * shear)
    return np.ascontiguousarray(np.stack(cols, axis=1))


def delayed_pressure(mesh, s_node, n_steps: int, dt: float, speed: float = 5.0,
                     harmonics: int = 5, period: float = 0.8, ramp_duration: float = 0.2):
    """Travelling-wave pressure p(t - s(x)/speed) in separable form.

    p(t - s/c) = a0 + sum_k a_k cos(k w t - k w s/c) = a0 + sum_k a_k [cos(k w t) cos(k w s/c)
    + sin(k w t) sin(k w s/c)], so the load is 1 + 2*harmonics spatial patterns times
    temporal amplitudes. s_node: [N] path length of each node from the inlet.
    Returns (modes [J][N][3], amp [n_steps][J]).
    """
    k = np.arange(1, harmonics + 1)
    w = 2 * np.pi / period
    grid = np.linspace(0.0, period, 200001)
    raw = np.sum(np.cos(w * k[None, :] * grid[:, None]) / k[None, :], axis=-1)
    lo, hi = raw.min(), raw.max()
    mean, half = 10.7e3, 2.7e3
    scale = 2.0 * half / (hi - lo)
    a0 = mean - half * (hi + lo) / (hi - lo)
    s_el = np.asarray(s_node, dtype=np.float64)[mesh.tri].mean(axis=1)
    pats = [np.ones(mesh.n_elems)]
    for kk in k:
        pats.append(np.cos(kk * w * s_el / speed))
        pats.append(np.sin(kk * w * s_el / speed))
    modes = pressure_shear_modes(mesh, delay_modes=pats)
    t = dt * np.arange(n_steps)
    r = ramp(t, ramp_duration)
    cols = [r * a0]
    for kk in k:
        ak = scale / kk
        cols.append(r * ak * np.cos(kk * w * t))
        cols.append(r * ak * np.sin(kk * w * t))
    return modes, np.ascontiguousarray(np.stack(cols, axis=1))


def peak_amplitudes(n_steps: int, dt: float, pressure: float = 13.4e3, shear: float = 1.0,
                    ramp_duration: float = 5.0e-3) -> np.ndarray:
    """Amplitude table [n_steps][2] holding the peak-systole pressure (10.7 + 2.7 kPa) and
    the axial shear after a quarter-sine ramp of `ramp_duration`."""
    t = dt * np.arange(n_steps)
    r = ramp(t, ramp_duration)
    return np.ascontiguousarray(np.stack([r * pressure, r * shear], axis=1))
