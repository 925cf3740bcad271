"""Pins of the per-sample coefficients and the assembled form.

* Three-point Gauss products (Section 2.2.1): the interior rule integrates the product
  of two linear fields exactly, so (E h)_e must equal the exact element average
  (sum_i E_i * sum_j h_j + sum_i E_i h_i) / 12 (the P1 mass-matrix identity), and hbar_e
  the mean of the corner thicknesses.
* Lumped mass (Section 2.3): total mass equals rho * sum_e A_e hbar_e, and for uniform
  thickness rho * h * (surface area).
* Assembly-free product (Section 2.4) equals the assembled CSR with 3 x 3 x S blocks
  (Section 2.3) and per-realisation scipy matrices.
* Statistics equal numpy's mean / var(ddof=1).
"""
import numpy as np
import pytest

import oracle
from oracle import assembled
import synth


def test_gauss_rule_exact_for_linear_products():
    case = synth.make_case("tube_small", S=3)
    m = case["mesh"]
    eh, hb = oracle.gauss_eh(m.tri, case["E"], case["h"])
    En = case["E"][m.tri]          # [E][3][S]
    hn = case["h"][m.tri]
    exact = (En.sum(1) * hn.sum(1) + (En * hn).sum(1)) / 12.0
    assert np.allclose(eh, exact, rtol=1e-14, atol=0)
    assert np.allclose(hb, hn.mean(1), rtol=1e-14, atol=0)


def test_lumped_mass_totals():
    case = synth.make_case("tube_small", S=2)
    mod = oracle.Model(case)
    total = mod.m_sn.sum(axis=1)
    expect = case["rho"] * (mod.area[None, :] * mod.hbar_se).sum(axis=1)
    assert np.allclose(total, expect, rtol=1e-13)
    uni = dict(case)
    uni["E"], uni["h"] = synth.lognormal_fields(case["mesh"], 1, uniform=True)
    mu = oracle.Model(uni)
    assert mu.m_sn.sum() == pytest.approx(case["rho"] * 1.0e-3 * mu.area.sum(), rel=1e-13)


def test_assembled_equals_matrix_free():
    case = synth.make_case("tube_small", S=3)
    mod = oracle.Model(case)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((mod.S, mod.N, 3)) * 1e-3
    f = mod.internal_force(u)
    row_ptr, col, blocks = assembled.block_csr(mod)
    y = assembled.block_csr_matvec(row_ptr, col, blocks, np.ascontiguousarray(u.transpose(1, 2, 0)))
    assert np.abs(y.transpose(2, 0, 1) - f).max() <= 1e-14 * np.abs(f).max() * 10
    for s in range(mod.S):
        K = assembled.assemble(mod, s)
        fs = K @ u[s].ravel()
        assert np.abs(fs - f[s].ravel()).max() <= 1e-13 * np.abs(fs).max()


def test_assembled_equals_matrix_free_tiny_tube(case_tiny):
    mod = oracle.Model(case_tiny, samples=[0, 5])
    rng = np.random.default_rng(9)
    u = rng.standard_normal((mod.S, mod.N, 3))
    f = mod.internal_force(u)
    for s in range(mod.S):
        fs = assembled.assemble(mod, s) @ u[s].ravel()
        assert np.linalg.norm(fs - f[s].ravel()) <= 1e-14 * np.linalg.norm(fs) * 10


def test_stats_match_numpy():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((33, 7, 3)) * 1e-3 + 0.5
    mean, var = oracle.stats(u)
    assert np.allclose(mean, u.mean(axis=0), rtol=1e-14, atol=0)
    assert np.allclose(var, u.var(axis=0, ddof=1), rtol=1e-12, atol=0)
    m1, v1 = oracle.stats(u[:1])
    assert np.array_equal(m1, u[0]) and np.all(v1 == 0)
