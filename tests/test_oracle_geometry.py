"""Pins of the geometry-updated oracle (oracle/geometry.py, Section 2.3 selective
re-assembly of K(u) on the deformed lumen).

* No re-assembly within the run (k beyond the last step) is the linear run, bit for bit.
* A rigid translation of the surface leaves every element matrix unchanged (to rounding).
* Static fixed point of a long clamped tube under internal pressure p (uniform E, h): on
  the deformed polygon of radius R + w the hoop strain of a radial displacement w is
  w / (R + w), while the lumped load stays p times the reference area; equilibrium
  E h w / ((1 - nu^2) R (R + w)) = p gives w = w_c / (1 - w_c / R) with the linear clamped
  value w_c = (1 - nu^2) p R^2 / (E h), whatever the re-assembly interval.

The reading K(X + u_m) u_n (total displacement times the stiffness of the deformed
surface) is not objective: a displacement-level contraction acts like a compressive
prestress. At the configuration's 10 kPa on the clamped tube (slopes near 0.2 rad in the
clamp boundary layers) and on an axially free tube (Poisson contraction) the oracle's
run leaves the fixed point and inverts elements within a few thousand steps; at the
paper's regime (displacements of the order of the wall thickness, small slopes) it
settles, which is where the pin is taken.
"""
import numpy as np
import pytest

import oracle
from oracle import geometry as og
import synth


def _uniform_case(mesh, n_steps, E=0.7e6, h=1.0e-3, p=1.0e4, alpha=1.0e3, S=1):
    En, hn = np.full((mesh.n_nodes, S), E), np.full((mesh.n_nodes, S), h)
    return dict(mesh=mesh, S=S, E=En, h=hn, rho=synth.configs.RHO, nu=synth.configs.NU,
                kshear=synth.configs.KSHEAR, alpha=alpha, dt=synth.cfl_dt(mesh, En),
                modes=synth.pressure_shear_modes(mesh), amp=synth.step_amplitudes(n_steps, p))


def _midspan_radial(mesh, u):
    nc, na = mesh.meta["nc"], mesh.meta["na"]
    ring = (na // 2) * nc + np.arange(nc)
    r = mesh.xyz[ring, :2]
    r = r / np.linalg.norm(r, axis=1)[:, None]
    return np.mean(np.einsum("ij,ij->i", u[ring, :2], r))


def test_no_reassembly_is_the_linear_run():
    case = synth.make_case("tube_small", S=3, n_steps=60, seed=1)
    lin = oracle.Model(case).run(50)[0]
    assert np.array_equal(og.run_updated(case, 50, 1000), lin)
    assert not np.array_equal(og.run_updated(case, 50, 10), lin)


def test_rigid_translation_leaves_element_matrices_unchanged():
    m = synth.tube_mesh(12, 8, length=0.03)
    K0, A0 = oracle.element_matrices(m.xyz, m.tri, 0.5, 5.0 / 6.0)
    K1, A1 = oracle.element_matrices(m.xyz + np.array([0.013, -0.2, 0.07]), m.tri, 0.5, 5.0 / 6.0)
    assert np.abs(K1 - K0).max() <= 1e-9 * np.abs(K0).max()
    assert np.abs(A1 - A0).max() <= 1e-9 * A0.max()


@pytest.mark.parametrize("k", [1, 25])
def test_fixed_point_matches_the_deformed_hoop_closed_form(k):
    """The paper's regime (displacements of the order of the wall thickness on slopes
    that stay small): p = 2 kPa on the clamped tube, w_c / R = 0.021. The ratio of the
    updated to the linear midspan displacement cancels the facet error of the mesh and
    must be 1 / (1 - w_c / R) = 1.0219 within a tenth of the effect, for re-assembly
    every step and every 25 steps alike."""
    R, E, h, p, nu = 0.01, 0.7e6, 1.0e-3, 2.0e3, synth.configs.NU
    m = synth.tube_mesh(48, 121, radius=R, length=0.3)
    n = 2400
    case = _uniform_case(m, n, E, h, p)
    w = _midspan_radial(m, og.run_updated(case, n, k)[0])
    lin = _midspan_radial(m, oracle.Model(case).run(n)[0][0])
    wc = (1 - nu * nu) * p * R * R / (E * h)
    assert lin == pytest.approx(wc, rel=0.01)
    effect = (wc / R) / (1 - wc / R)
    assert w / lin - 1.0 == pytest.approx(effect, rel=0.1)
