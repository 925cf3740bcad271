"""Pins of the output-statistics oracle: order statistics and the type-7 definition,
numpy's independent quantile and variance routines, and closed-form stress states of a
straight tube (uniform axial stretch, uniform radial expansion, twist), zero stress under
the shell's rigid modes, and invariance of the cylindrical components under a rigid
rotation of the whole problem."""
import numpy as np
import pytest

import oracle.outputs as oo
import synth

NU, KS, E0 = 0.5, 5.0 / 6.0, 0.7e6


def test_quantiles_are_order_statistics_at_grid_probabilities():
    rng = np.random.Generator(np.random.Philox(key=1))
    rows = rng.standard_normal((5, 9))
    q = [k / 8 for k in range(9)]
    Q = oo.quantiles(rows, q)
    assert np.array_equal(Q, np.sort(rows, axis=1))


def test_quantiles_interpolate_linearly_and_match_numpy():
    assert oo.quantiles(np.array([[0.0, 10.0]]), [0.25, 0.5, 0.9])[0].tolist() == [2.5, 5.0, 9.0]
    rng = np.random.Generator(np.random.Philox(key=2))
    for S in (1, 2, 7, 64, 201):
        rows = rng.standard_normal((4, S)) * 3.0 + 1.0
        q = [0.0, 0.05, 0.5, 0.95, 1.0, 0.333]
        Q = oo.quantiles(rows, q)
        ref = np.quantile(rows, q, axis=1, method="linear").T
        assert np.allclose(Q, ref, rtol=0, atol=1e-14 * np.abs(rows).max())
        perm = rng.permutation(S)
        assert np.array_equal(oo.quantiles(rows[:, perm], q), Q)   # order of samples is irrelevant
        assert np.all(np.diff(oo.quantiles(rows, np.linspace(0, 1, 11)), axis=1) >= 0)


def test_row_stats_match_numpy():
    rng = np.random.Generator(np.random.Philox(key=3))
    rows = rng.standard_normal((6, 33)) * 1e-5 + 2e-5
    m, v, _ = oo.row_stats(rows)
    assert np.allclose(m, rows.mean(axis=1), rtol=1e-14)
    assert np.allclose(v, rows.var(axis=1, ddof=1), rtol=1e-12)
    m1, v1, q1 = oo.row_stats(rows[:, :1], [0.5])
    assert np.array_equal(v1, np.zeros(6)) and np.array_equal(q1[:, 0], rows[:, 0])


def _tube(nc=24, na=9, R=0.01, L=0.04):
    m = synth.tube_mesh(nc=nc, na=na, radius=R, length=L)
    cl = np.array([[0.0, 0.0, -0.01], [0.0, 0.0, L + 0.01]])
    return m, cl


def _stress(m, u_nc, E=E0, cl=None):
    S = 1
    E_node = np.full((m.n_nodes, S), E)
    return oo.element_stress(m.xyz, m.tri, u_nc[None], E_node, NU, KS, cl).reshape(-1, 6)


def test_uniform_axial_stretch():
    m, cl = _tube()
    eps = 1e-4
    u = np.zeros((m.n_nodes, 3))
    u[:, 2] = eps * m.xyz[:, 2]
    s = _stress(m, u, cl=cl)
    f = E0 / (1 - NU * NU)
    scale = f * eps
    assert np.allclose(s[:, 2], f * eps, rtol=1e-12)            # zz
    assert np.allclose(s[:, 1], NU * f * eps, rtol=1e-12)       # theta theta
    assert np.abs(s[:, [0, 3, 4, 5]]).max() < 1e-12 * scale     # rr and shears


def test_uniform_radial_expansion():
    m, cl = _tube()
    eps = 2e-4
    u = np.zeros((m.n_nodes, 3))
    u[:, :2] = eps * m.xyz[:, :2]
    s = _stress(m, u, cl=cl)
    f = E0 / (1 - NU * NU)
    assert np.allclose(s[:, 1], f * eps, rtol=1e-12)
    assert np.allclose(s[:, 2], NU * f * eps, rtol=1e-12)
    assert np.abs(s[:, [0, 3, 4, 5]]).max() < 1e-12 * f * eps


def test_twist_gives_the_in_plane_shear():
    """u = phi z (-y, x, 0): shear strain phi R along (circumferential, axial); with the
    frame's theta = r x z (opposite to the usual circumferential sense) the sign flips."""
    m, cl = _tube(nc=96, na=41, L=0.04)
    phi = 1e-3
    u = np.zeros((m.n_nodes, 3))
    u[:, 0] = -phi * m.xyz[:, 2] * m.xyz[:, 1]
    u[:, 1] = phi * m.xyz[:, 2] * m.xyz[:, 0]
    s = _stress(m, u, cl=cl)
    ref = -E0 / (2 * (1 + NU)) * phi * 0.01
    assert np.allclose(s[:, 5], ref, rtol=2e-3)
    assert np.abs(s[:, [0, 1, 2]]).max() < 1e-2 * abs(ref)


def test_rigid_modes_are_stress_free():
    m = synth.aneurysm_mesh(nc=20, na=16)
    cl = np.array([[0.0, 0.0, -0.01], [0.0, 0.0, 0.13]])
    rng = np.random.Generator(np.random.Philox(key=4))
    t = rng.standard_normal(3) * 1e-4
    u = np.tile(t, (m.n_nodes, 1))
    s = _stress(m, u, cl=cl)
    ref = E0 * 1e-4
    assert np.abs(s).max() < 1e-10 * ref


def test_components_invariant_under_rigid_rotation():
    m = synth.aneurysm_mesh(nc=20, na=16)
    cl = np.stack([np.zeros(30), np.zeros(30), np.linspace(-0.01, 0.13, 30)], axis=1)
    rng = np.random.Generator(np.random.Philox(key=5))
    S = 3
    u = rng.standard_normal((S, m.n_nodes, 3)) * 1e-5
    E_node = E0 * np.exp(0.1 * rng.standard_normal((m.n_nodes, S)))
    a = oo.element_stress(m.xyz, m.tri, u, E_node, NU, KS, cl)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    b = oo.element_stress(m.xyz @ Q.T, m.tri, u @ Q.T, E_node, NU, KS, cl @ Q.T)
    assert np.abs(a - b).max() < 1e-9 * np.abs(a).max()
