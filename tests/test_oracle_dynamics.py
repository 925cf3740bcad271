"""Pins of the oracle's time stepping and of the model it integrates.

* Hoop closed forms (thin cylinder under internal pressure p, uniform E and h):
  axially free ends give u_r = p R^2 / (E h); clamped ends (eps_z ~ 0 away from the
  ends) give u_r = (1 - nu^2) p R^2 / (E h). Checked on the static solution of the
  assembled system, which pins element matrices and load patterns together.
* Radial breathing frequency of a clamped thin cylinder, omega^2 = E / (rho (1 - nu^2) R^2):
  the discrete generalised eigenvalue of (K, M) closest to it is within 3 %.
* Exact modal solution of the central-difference recursion: started from a discrete
  eigenvector phi with zero velocity and no load, the undamped scheme must give
  u_n = phi cos(n theta) with cos(theta) = 1 - omega^2 dt^2 / 2, and the damped scheme the
  characteristic-root solution; this pins the start and every term of Eq. (dynamicsCD).
* Second-order convergence to the continuous damped oscillator as dt is halved.
* Discrete energy H_n = 1/2 d^T (M/dt^2 - K/4) d + 1/2 w^T K w - f^T w, with d = u_{n+1} - u_n
  and w = (u_n + u_{n+1}) / 2, is conserved by the undamped scheme under constant load.
* Static limit: the damped run converges to the direct solve K_s u = f per realisation.
* Ensemble invariants: realisations are independent systems, so permuting them permutes
  the trajectories, a one-member run equals that member of the ensemble, and uniform
  fields give identical members whose tube response is axisymmetric (no circumferential
  displacement, Section 3.1's homogeneous case).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import oracle
from oracle import assembled
import synth


def _uniform_case(mesh, E=0.7e6, h=1.0e-3, p=1.0e4, alpha=0.0, n_steps=10, dt=None):
    S = 1
    En, hn = np.full((mesh.n_nodes, S), E), np.full((mesh.n_nodes, S), h)
    case = dict(mesh=mesh, S=S, E=En, h=hn, rho=synth.configs.RHO, nu=synth.configs.NU,
                kshear=synth.configs.KSHEAR, alpha=alpha,
                dt=dt if dt is not None else synth.cfl_dt(mesh, En),
                modes=synth.pressure_shear_modes(mesh), amp=synth.step_amplitudes(n_steps, p))
    return case


def _static(mod, case, sample=0):
    K = assembled.assemble(mod, sample).tocsc()
    f = (case["modes"][0] * case["amp"][0, 0]).ravel()
    free = np.flatnonzero(mod.fixed == 0)
    u = np.zeros(3 * mod.N)
    u[free] = spla.spsolve(K[free][:, free], f[free])
    return u.reshape(mod.N, 3)


def _midspan_radial(mesh, u):
    nc, na = mesh.meta["nc"], mesh.meta["na"]
    ring = (na // 2) * nc + np.arange(nc)
    r = mesh.xyz[ring, :2]
    r = r / np.linalg.norm(r, axis=1)[:, None]
    return np.mean(np.einsum("ij,ij->i", u[ring, :2], r))


def test_hoop_axially_free():
    R, E, h, p, nu = 0.01, 0.7e6, 1.0e-3, 1.0e4, synth.configs.NU
    m = synth.tube_mesh(64, 33, radius=R, length=0.1, clamp_ends=False)
    nc = m.meta["nc"]
    m.fixed[:nc, 2] = 1                         # bottom ring: axial dof only
    m.fixed[0, 1] = 1                           # theta = 0: tangential (y)
    m.fixed[nc // 4, 0] = 1                     # theta = 90 deg: tangential (x)
    m.fixed[nc // 2, 1] = 1
    m.fixed[3 * nc // 4, 0] = 1
    case = _uniform_case(m, E, h, p)
    mod = oracle.Model(case)
    ur = _midspan_radial(m, _static(mod, case))
    assert ur == pytest.approx(p * R * R / (E * h), rel=0.01)


def test_hoop_clamped():
    R, E, h, p, nu = 0.01, 0.7e6, 1.0e-3, 1.0e4, synth.configs.NU
    # Long tube: with both ends clamped the mean axial strain is zero, so eps_z at
    # midspan is -nu * eps_theta * (boundary-layer length / L); at L = 40 R it is < 1 %.
    m = synth.tube_mesh(64, 161, radius=R, length=0.4)
    case = _uniform_case(m, E, h, p)
    mod = oracle.Model(case)
    ur = _midspan_radial(m, _static(mod, case))
    assert ur == pytest.approx((1 - nu * nu) * p * R * R / (E * h), rel=0.01)
    # the wrong Gauss-weight normalisation (weights summing to 1/2) would double u_r
    assert abs(ur / ((1 - nu * nu) * p * R * R / (E * h)) - 2.0) > 0.5


def _free_dense(mod, sample=0):
    K = assembled.assemble(mod, sample).toarray()
    Mv = assembled.lumped_mass_vector(mod, sample)
    free = np.flatnonzero(mod.fixed == 0)
    return K[np.ix_(free, free)], Mv[free], free


def test_breathing_frequency_clamped():
    R, E, h, nu = 0.01, 0.7e6, 1.0e-3, synth.configs.NU
    m = synth.tube_mesh(32, 41, radius=R, length=0.1)
    mod = oracle.Model(_uniform_case(m, E, h))
    Kf, Mf, free = _free_dense(mod)
    lam, phi = sla.eigh(Kf, np.diag(Mf))
    radial = np.zeros((m.n_nodes, 3))
    radial[:, :2] = m.xyz[:, :2] / np.linalg.norm(m.xyz[:, :2], axis=1)[:, None]
    r = radial.ravel()[free]
    proj = np.abs(phi.T @ (Mf * r)) / np.sqrt(np.einsum("ij,i,ij->j", phi, Mf, phi) * (r @ (Mf * r)))
    k = int(np.argmax(proj))
    omega0 = np.sqrt(E / (synth.configs.RHO * (1 - nu * nu))) / R
    assert np.sqrt(lam[k]) == pytest.approx(omega0, rel=0.03)


def _mode_case(alpha, dt, n):
    m = synth.tube_mesh(12, 8, length=0.03)
    case = _uniform_case(m, alpha=alpha, n_steps=n, dt=dt)
    case["amp"] = np.zeros((n, 1))
    mod = oracle.Model(case)
    Kf, Mf, free = _free_dense(mod)
    lam, phi = sla.eigh(Kf, np.diag(Mf))
    k = len(lam) // 3
    u0 = np.zeros(3 * mod.N)
    u0[free] = phi[:, k] / np.abs(phi[:, k]).max() * 1e-3
    return mod, lam[k], u0.reshape(1, mod.N, 3)


@pytest.mark.parametrize("alpha", [0.0, 800.0])
def test_modal_solution_is_exact(alpha):
    n = 400
    mod, lam, u0 = _mode_case(alpha, 2.0e-6, n)
    dt = mod.dt
    up, uc = mod.start(u0=u0)
    beta = 0.5 * alpha * dt
    r = np.sqrt((1 - beta) / (1 + beta))
    cth = (2 - lam * dt * dt) / (2 * (1 + beta) * r)
    th = np.arccos(cth)
    xm1 = 1 - 0.5 * lam * dt * dt
    c = (np.cos(th) - r * xm1) / np.sin(th)
    errs = []
    for step in range(0, n, 100):
        mod.steps(up, uc, step, 100)
        nn = step + 100
        x = r ** nn * (np.cos(nn * th) + c * np.sin(nn * th))
        errs.append(np.abs(uc - x * u0).max() / np.abs(u0).max())
    assert max(errs) < 1e-9


def test_second_order_convergence_to_continuous_oscillator():
    alpha, T = 800.0, 4.0e-4
    errs = []
    for dt in (2.0e-6, 1.0e-6):
        n = int(round(T / dt))
        mod, lam, u0 = _mode_case(alpha, dt, n)
        up, uc = mod.start(u0=u0)
        mod.steps(up, uc, 0, n)
        wd = np.sqrt(lam - 0.25 * alpha * alpha)
        x = np.exp(-0.5 * alpha * T) * (np.cos(wd * T) + 0.5 * alpha / wd * np.sin(wd * T))
        errs.append(np.abs(uc - x * u0).max() / np.abs(u0).max())
    assert errs[1] < errs[0]
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


def test_energy_conserved_undamped():
    case = synth.make_case("tube_small", S=2, n_steps=2000, alpha=0.0)
    mod = oracle.Model(case)
    up, uc = mod.start()
    f = (case["modes"][0] * case["amp"][0, 0]).ravel()
    Hs, scale = [], []
    for chunk in range(10):
        mod.steps(up, uc, chunk * 200, 200)
        # (up, uc) = (u_n, u_{n+1}) for n = 200 (chunk + 1) - 1
        for s in range(mod.S):
            K = assembled.assemble(mod, s)
            Mv = assembled.lumped_mass_vector(mod, s)
            d = (uc[s] - up[s]).ravel()
            w = 0.5 * (uc[s] + up[s]).ravel()
            kin = 0.5 * d @ (Mv * d) / mod.dt ** 2 - 0.125 * d @ (K @ d)
            pot = 0.5 * w @ (K @ w)
            Hs.append((s, kin + pot - f @ w))
            scale.append(abs(kin) + abs(pot) + abs(f @ w))
    for s in range(mod.S):
        H = np.array([h for (ss, h) in Hs if ss == s])
        assert np.abs(H - H[0]).max() <= 1e-10 * max(scale)
    assert max(scale) > 0


@pytest.mark.slow
def test_static_limit_of_damped_run(case_tiny):
    mod = oracle.Model(case_tiny, samples=[0, 3, 7])
    n = 12000
    mod.amp = np.ascontiguousarray(np.repeat(case_tiny["amp"][:1], n, axis=0))
    u, _ = mod.run(n)
    for k in range(mod.S):
        us = _static(mod, dict(case_tiny, amp=mod.amp), sample=k)
        assert np.linalg.norm(u[k] - us) <= 1e-7 * np.linalg.norm(us)


def test_ensemble_invariants():
    """A sample index mixed into another sample's coefficients (a transposed [N][S] field,
    a shared mass, a wrong stride) breaks one of these, all of which hold bit for bit."""
    case = synth.make_case("tube_small", S=4, n_steps=80, seed=2)
    u = oracle.Model(case).run(60)[0]                       # [S][N][3]
    perm = [2, 0, 3, 1]
    shuffled = dict(case, E=case["E"][:, perm], h=case["h"][:, perm])
    assert np.array_equal(oracle.Model(shuffled).run(60)[0], u[perm])
    assert np.array_equal(oracle.Model(case, samples=[3]).run(60)[0][0], u[3])
    # uniform fields: identical members, axisymmetric response of the clamped tube
    from synth.configs import _case
    m = synth.tube_mesh(24, 20, length=0.06)
    uni = _case(m, 3, 0, 400, "step", uniform=True)
    uu = oracle.Model(uni).run(300)[0]
    assert np.array_equal(uu[0], uu[1]) and np.array_equal(uu[0], uu[2])
    x = m.xyz
    r = np.hypot(x[:, 0], x[:, 1])
    u_r = (uu[0, :, 0] * x[:, 0] + uu[0, :, 1] * x[:, 1]) / r
    u_t = (-uu[0, :, 0] * x[:, 1] + uu[0, :, 1] * x[:, 0]) / r
    assert np.abs(u_r).max() > 0
    assert np.abs(u_t).max() <= 1e-12 * np.abs(u_r).max()

