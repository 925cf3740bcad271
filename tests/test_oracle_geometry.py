"""Pins of the geometry-updated oracle (oracle/geometry.py, Section 2.3: the stiffness of
the current surface, re-assembled every k steps, applied to displacement increments).

* No re-assembly within the run (k beyond the last step) is the linear run, bit for bit.
* A rigid translation of the surface leaves every element matrix unchanged (to rounding).
* The stiffness of a deformed tube: on the polygon of radius R + w (a uniform radial
  displacement of a straight tube), a radial increment stretches the hoop by
  1 / (R + w) instead of 1 / R, so the midspan radial force of the re-assembled element
  matrices is R / (R + w) times the reference one, exactly.
* Static fixed point of a long clamped tube under internal pressure p (uniform E, h):
  the hoop force accumulated along the path is E h / (1 - nu^2) * ln((R + w) / R) and
  balances the reference-area load p R, so w = R (exp(w_c / R) - 1) with the linear clamped
  value w_c = (1 - nu^2) p R^2 / (E h). With re-assembly every step the damped run settles
  at that ratio to the linear run (within a tenth of the effect, which the mesh's facet
  error cancels out of the ratio); K(X + u) u_total would settle at 1 / (1 - w_c / R).
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


def test_reassembled_hoop_stiffness_of_a_deformed_tube():
    R = 0.01
    m = synth.tube_mesh(48, 121, radius=R, length=0.3)
    case = _uniform_case(m, 2)
    mod = oracle.Model(case)
    rhat = np.zeros((m.n_nodes, 3))
    rhat[:, :2] = m.xyz[:, :2] / np.linalg.norm(m.xyz[:, :2], axis=1)[:, None]
    ring = (m.meta["na"] // 2) * m.meta["nc"] + np.arange(m.meta["nc"])

    def radial_force(w):
        K, _ = oracle.element_matrices(m.xyz + w * rhat, m.tri, case["nu"], case["kshear"])
        mod.Kg = np.ascontiguousarray(K.reshape(mod.E, 81))
        f = mod.internal_force(1e-6 * rhat[None])[0]
        return np.mean(np.einsum("ij,ij->i", f[ring], rhat[ring]))

    f0 = radial_force(0.0)
    for w in (1e-4, 1e-3):
        assert radial_force(w) / f0 == pytest.approx(R / (R + w), rel=1e-9)


def test_fixed_point_matches_the_accumulated_hoop_closed_form():
    """The paper's regime: p = 2 kPa on the clamped tube, w_c / R = 0.021; re-assembly
    every step (selective re-assembly adds a path bias of order k: the stiffness of a
    segment's start is used for its whole loading or unloading)."""
    R, E, h, p, nu = 0.01, 0.7e6, 1.0e-3, 2.0e3, synth.configs.NU
    m = synth.tube_mesh(48, 121, radius=R, length=0.3)
    n = 2400
    case = _uniform_case(m, n, E, h, p)
    w = _midspan_radial(m, og.run_updated(case, n, 1)[0])
    lin = _midspan_radial(m, oracle.Model(case).run(n)[0][0])
    wc = (1 - nu * nu) * p * R * R / (E * h)
    assert lin == pytest.approx(wc, rel=0.01)
    x = wc / R
    assert w / lin - 1.0 == pytest.approx((np.exp(x) - 1.0) / x - 1.0, rel=0.1)
