"""Pins of the running-peak oracle (oracle/outputs.py peak_magnitude).

* Brute force: the peak over the recorded steps equals the largest |u_k| of independent
  runs from rest to every recorded step k (a different route: every u_k is recomputed
  from the start, with no running state).
* Dynamic amplification of a step load on one mode: a load f = M phi on a discrete
  eigenvector (K phi = lambda M phi) applied from rest excites that mode alone, so
  u_n = (phi / lambda) (1 - x_n) exactly, with x_n the mode's free response from a unit
  displacement: cos(n theta) undamped, r^n (cos n theta + c sin n theta) damped (the
  characteristic roots of the recursion, as in the modal pin of the time stepping). The
  peak magnitude of node i is therefore |phi_i| / lambda * max_k |1 - x_k| over the
  recorded steps k: about twice the static value when undamped (the classical factor of
  two), less when damped. A peak of a single dof instead of the nodal magnitude, a
  minimum, a last value or a wrong recording step all fail it.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import assembled
from oracle import outputs as oo
import synth


def test_peak_equals_brute_force_over_fresh_runs():
    case = synth.make_case("plate", S=3, n_steps=40, seed=4)
    mod = oracle.Model(case)
    n = 24
    for stride in (1, 5):
        peak, _, uc = oo.peak_magnitude(mod, n, stride)
        ks = [k for k in range(1, n + 1) if k % stride == 0]
        brute = np.max([oo.magnitude_rows(mod.run(k)[0]) for k in ks], axis=0)
        assert np.array_equal(peak, brute), stride
        assert np.array_equal(uc, mod.run(n)[0])
    # continuing from a saved state gives the same peak as one long run
    p1, up, uc = oo.peak_magnitude(mod, 10, 5)
    p2, _, _ = oo.peak_magnitude(mod, 14, 5, up=up, uc=uc, step0=10, peak=p1)
    assert np.array_equal(p2, oo.peak_magnitude(mod, 24, 5)[0])


@pytest.mark.parametrize("alpha", [0.0, 800.0])
@pytest.mark.parametrize("stride", [1, 7])
def test_peak_of_a_single_mode_step_response(alpha, stride):
    m = synth.tube_mesh(12, 8, length=0.03)
    S = 1
    En, hn = np.full((m.n_nodes, S), 0.7e6), np.full((m.n_nodes, S), 1.0e-3)
    n = 600
    case = dict(mesh=m, S=S, E=En, h=hn, rho=synth.configs.RHO, nu=synth.configs.NU,
                kshear=synth.configs.KSHEAR, alpha=alpha, dt=2.0e-6,
                modes=np.zeros((1, m.n_nodes, 3)), amp=np.ones((n, 1)))
    mod = oracle.Model(case)
    K = assembled.assemble(mod, 0).toarray()
    Mv = assembled.lumped_mass_vector(mod, 0)
    free = np.flatnonzero(mod.fixed == 0)
    lam, phi = sla.eigh(K[np.ix_(free, free)], np.diag(Mv[free]))
    k = len(lam) // 4
    ph = np.zeros(3 * mod.N)
    ph[free] = phi[:, k] / np.abs(phi[:, k]).max()
    lam = lam[k]
    mod.modes = np.ascontiguousarray((Mv * ph).reshape(1, mod.N, 3) * 1e-3 * lam)  # u_static = 1e-3 phi
    peak, _, _ = oo.peak_magnitude(mod, n, stride)
    dt = mod.dt
    beta = 0.5 * alpha * dt
    r = np.sqrt((1 - beta) / (1 + beta))
    th = np.arccos((2 - lam * dt * dt) / (2 * (1 + beta) * r))
    c = (np.cos(th) - r * (1 - 0.5 * lam * dt * dt)) / np.sin(th)
    ks = np.arange(stride, n + 1, stride)
    x = r ** ks * (np.cos(ks * th) + c * np.sin(ks * th))
    amp = np.abs(1.0 - x).max()
    node_static = 1e-3 * np.linalg.norm(ph.reshape(mod.N, 3), axis=1)
    expect = node_static * amp
    assert np.abs(peak[:, 0] - expect).max() <= 1e-9 * expect.max()
    if alpha == 0.0:
        assert amp == pytest.approx(2.0, abs=0.02)     # the factor of two of a step load
    else:
        assert 1.0 < amp < 1.9
