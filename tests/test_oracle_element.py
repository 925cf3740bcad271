"""Pins of the oracle's element stiffness (Section 2.2.1: B, C, k_e).

Each check is fixed by mechanics, not by re-typing the oracle's formula:
  * symmetry and positive semi-definiteness of A B^T C B;
  * the null space is exactly the rigid motions a 3-dof shell element without rotation
    dofs cannot feel: three translations and the in-plane rotation (4 zero eigenvalues);
    the out-of-plane rotations strain the transverse shear terms and must cost energy;
  * invariance under relabelling the corners (which changes the local e1 axis) and under
    a rigid rotation of the element;
  * membrane and transverse-shear patch tests on a jittered flat plate: a linear
    displacement field gives zero force at interior nodes and strain energy
    area * (E h) * eps^T C0 eps.
A dropped term in B, a wrong sign in x_ij, or a transposed rotation fails one of these.
"""
import numpy as np
import pytest

import oracle
import synth

NU, KS = 0.5, 5.0 / 6.0


def _rot(axis, ang):
    axis = np.asarray(axis, float)
    axis /= np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


X0 = synth.single_triangle().xyz


def test_symmetric_psd_four_zero_modes():
    K, A = oracle.element_matrix(X0, NU, KS)
    assert A > 0
    assert np.allclose(K, K.T, rtol=0, atol=1e-13 * np.abs(K).max())
    w = np.linalg.eigvalsh(K)
    lmax = w.max()
    assert w.min() > -1e-12 * lmax
    assert np.sum(np.abs(w) < 1e-12 * lmax) == 4
    assert np.sum(w > 1e-8 * lmax) == 5


def test_null_space_is_translations_and_inplane_rotation():
    K, _ = oracle.element_matrix(X0, NU, KS)
    scale = np.abs(K).max()
    for d in range(3):
        t = np.zeros(9)
        t[d::3] = 1.0
        assert np.abs(K @ t).max() < 1e-12 * scale
    n = np.cross(X0[1] - X0[0], X0[2] - X0[0])
    n /= np.linalg.norm(n)
    c = X0.mean(axis=0)
    rot_n = np.concatenate([np.cross(n, X0[j] - c) for j in range(3)])
    assert np.abs(K @ rot_n).max() < 1e-12 * scale * np.linalg.norm(rot_n)
    # out-of-plane rotation about an in-plane axis bends the element: positive energy
    e1 = (X0[1] - X0[0]) / np.linalg.norm(X0[1] - X0[0])
    rot_t = np.concatenate([np.cross(e1, X0[j] - c) for j in range(3)])
    assert rot_t @ K @ rot_t > 1e-6 * scale * (rot_t @ rot_t)


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 0, 1)])
def test_corner_relabelling_invariance(perm):
    K, _ = oracle.element_matrix(X0, NU, KS)
    Kp, _ = oracle.element_matrix(X0[list(perm)], NU, KS)
    idx = np.concatenate([3 * p + np.arange(3) for p in perm])
    assert np.allclose(Kp, K[np.ix_(idx, idx)], rtol=0, atol=1e-13 * np.abs(K).max())


def test_rigid_rotation_covariance():
    K, _ = oracle.element_matrix(X0, NU, KS)
    R = _rot([0.3, -0.5, 0.8], 0.77)
    Kr, _ = oracle.element_matrix((R @ X0.T).T + np.array([0.1, -0.2, 0.05]), NU, KS)
    Rb = np.kron(np.eye(3), R)
    assert np.allclose(Kr, Rb @ K @ Rb.T, rtol=0, atol=1e-13 * np.abs(K).max())


def _plate_model():
    m = synth.plate_mesh(6, 5, jitter=0.25, seed=3)
    case = dict(mesh=m, E=np.full((m.n_nodes, 1), 2.0e6), h=np.full((m.n_nodes, 1), 1.5e-3),
                nu=NU, kshear=KS, rho=1000.0, alpha=0.0, dt=1e-6,
                modes=np.zeros((1, m.n_nodes, 3)), amp=np.zeros((2, 1)))
    return m, oracle.Model(case)


def _interior(m):
    nx, ny = m.meta["nx"], m.meta["ny"]
    ii = []
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            ii.append(j * nx + i)
    return np.array(ii)


def test_membrane_patch_test():
    m, mod = _plate_model()
    G = np.array([[1.3e-3, -0.4e-3], [0.7e-3, -0.9e-3]])   # du_i/dx_j, in-plane
    u = np.zeros((m.n_nodes, 3))
    u[:, :2] = m.xyz[:, :2] @ G.T
    f = mod.internal_force(u[None])[0]
    scale = np.abs(f).max()
    assert scale > 0
    assert np.abs(f[_interior(m)]).max() < 1e-11 * scale
    eps = np.array([G[0, 0], G[1, 1], G[0, 1] + G[1, 0]])
    c = 1.0 / (1 - NU ** 2)
    C0 = c * np.array([[1, NU, 0], [NU, 1, 0], [0, 0, 0.5 * (1 - NU)]])
    area = mod.area.sum()
    Eh = 2.0e6 * 1.5e-3
    energy = 0.5 * (u.ravel() @ f.ravel())
    assert energy == pytest.approx(0.5 * area * Eh * eps @ C0 @ eps, rel=1e-12)


def test_transverse_shear_patch_test():
    m, mod = _plate_model()
    a, b = 2.0e-3, -1.1e-3
    u = np.zeros((m.n_nodes, 3))
    u[:, 2] = a * m.xyz[:, 0] + b * m.xyz[:, 1]
    f = mod.internal_force(u[None])[0]
    assert np.abs(f[_interior(m)]).max() < 1e-11 * np.abs(f).max()
    g = KS * 0.5 * (1 - NU) / (1 - NU ** 2)
    energy = 0.5 * (u.ravel() @ f.ravel())
    assert energy == pytest.approx(0.5 * mod.area.sum() * 2.0e6 * 1.5e-3 * g * (a * a + b * b), rel=1e-12)
