"""Checks of the synthetic input generators (not of the solver).

* Random fields (Section 2.1): interior marginal standard deviation matches the target
  within Monte-Carlo error, and the empirical correlation at the correlation length is
  close to the Matern value there (about 0.1, Eq. 1).
* Pressure patterns: the resultant radial force on a tube equals p times its lateral
  (polygonal) area and the net force vanishes by symmetry.
* The stable step rule reproduces the paper's printed back-of-the-envelope numbers
  (tests/golden/paper_cfl_example.json).
"""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mesh_orientation_and_counts():
    m = synth.tube_mesh(40, 40)
    assert m.n_nodes == 1600 and m.n_elems == 3120
    X = m.xyz[m.tri]
    n = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    c = X.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", n[:, :2], c[:, :2]) > 0)
    a = synth.aneurysm_mesh(40, 50)
    assert a.xyz[:, :2].max() <= 0.02 + 1e-12


def test_field_marginal_std_and_correlation():
    m = synth.tube_mesh(48, 72, length=0.15)
    S = 200
    (g,) = synth.fields.gmrf_fields(m.xyz, m.tri, S, 0.02, 0.1, seed=11, streams=(1,))
    nc, na = 48, 72
    rings = np.arange(na)
    inner = np.concatenate([r * nc + np.arange(nc) for r in rings[na // 4: 3 * na // 4]])
    sd = g[inner].std(axis=1, ddof=1)
    # mesh-level GMRF variance matches the continuum value to within a few percent
    assert np.mean(sd) == pytest.approx(0.1, rel=0.08)
    # correlation between nodes one correlation length apart along the axis
    dz = m.xyz[nc, 2] - m.xyz[0, 2]
    k = int(round(0.02 / dz))
    a = inner[inner + k * nc < m.n_nodes]
    rho = np.mean([np.corrcoef(g[i], g[i + k * nc])[0, 1] for i in a[:: 7]])
    d = m.xyz[k * nc, 2] - m.xyz[0, 2]
    assert rho == pytest.approx(float(synth.matern_correlation(d, 0.02)), abs=0.08)


def test_independent_streams_and_seeds():
    m = synth.tube_mesh(12, 8, length=0.03)
    E1, h1 = synth.lognormal_fields(m, 4, seed=3)
    E2, h2 = synth.lognormal_fields(m, 4, seed=3)
    assert np.array_equal(E1, E2) and np.array_equal(h1, h2)
    gE, gh = np.log(E1 / 0.7e6), np.log(h1 / 1e-3)
    assert abs(np.corrcoef(gE.ravel(), gh.ravel())[0, 1]) < 0.5


def test_pressure_resultant():
    m = synth.tube_mesh(40, 20, clamp_ends=False)
    P = synth.pressure_shear_modes(m)[0]
    assert np.abs(P.sum(axis=0)).max() < 1e-15
    X = m.xyz[m.tri]
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1).sum()
    assert np.linalg.norm(P, axis=1).sum() == pytest.approx(area, rel=0.02)


def test_cfl_rule_matches_paper_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_cfl_example.json")))
    # one equilateral triangle whose inscribed circle has diameter l_min
    side = g["l_min_m"] * np.sqrt(3.0)
    pts = [[0, 0, 0], [side, 0, 0], [side / 2, side * np.sqrt(3) / 2, 0]]
    m = synth.single_triangle(pts)
    dt = synth.cfl_dt(m, np.array([g["E_pa"]]), rho=g["rho_printed"], safety=1.0)
    assert dt == pytest.approx(g["dt_printed_s"], rel=0.05)
    assert g["safety"] * dt == pytest.approx(g["dt_after_safety_printed_s"], rel=0.15)


def test_cylinder_workload_follows_section_3_1():
    """The paper's cylinder: D = 4 cm, L = 30 cm, the three mesh densities' triangle counts,
    Gaussian fields with the stated means and standard deviations, 13 mmHg plus the steady
    Poiseuille load (pressure drop 8 mu L Q / (pi R^4), wall shear 4 mu Q / (pi R^3))."""
    import numpy as np
    import synth
    for level, n_tri in ((0, 5074), (1, 15136), (2, 32994)):
        c = synth.make_case("cylinder", level=level, S=2, n_steps=3, host_fields=False)
        m = c["mesh"]
        assert m.n_elems == n_tri
        r = np.hypot(m.xyz[:, 0], m.xyz[:, 1])
        assert np.allclose(r, 0.02) and m.xyz[:, 2].min() == 0.0 and np.isclose(m.xyz[:, 2].max(), 0.30)
    c = synth.make_case("cylinder", level=0, S=400, corr=0.0095, n_steps=20000, seed=5)
    E, h = c["E"], c["h"]
    assert abs(E.mean() / 0.7e6 - 1) < 0.02 and abs(E.std() / 0.07e6 - 1) < 0.15
    assert abs(h.mean() / 4e-3 - 1) < 0.02 and abs(h.std() / 0.4e-3 - 1) < 0.15
    mu, Q, R, L = 4e-3, 66.59e-6, 0.02, 0.30
    amp = c["amp"][-1]                                   # after the ramp
    assert np.isclose(amp[0], 13 * 133.322387415)
    assert np.isclose(amp[1], 8 * mu * L * Q / (np.pi * R ** 4))
    assert np.isclose(amp[2], 4 * mu * Q / (np.pi * R ** 3))
    # pattern 1 carries the linear drop: total force of the pressure patterns is radial
    # (zero resultant), and pattern 1 weighs the inlet end more than the outlet end
    P1 = c["modes"][1]
    m = c["mesh"]
    inlet = m.xyz[:, 2] < 0.05
    outlet = m.xyz[:, 2] > 0.25
    assert np.linalg.norm(P1[inlet], axis=1).mean() > 3 * np.linalg.norm(P1[outlet], axis=1).mean()


def test_shards_of_one_ensemble_are_its_realisations():
    """Realisations are keyed by their index in the seeded ensemble, so a rank that draws
    realisations [k, k + S) gets those of the whole ensemble (sample-sharded runs)."""
    whole = synth.make_case("tube_small", S=6, seed=3)
    for k in (0, 2, 5):
        part = synth.make_case("tube_small", S=6 - k, seed=3, sample0=k)
        assert np.allclose(part["E"], whole["E"][:, k:], rtol=1e-14, atol=0)
        assert np.allclose(part["h"], whole["h"][:, k:], rtol=1e-14, atol=0)
