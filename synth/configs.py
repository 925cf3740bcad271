"""Named synthetic workloads and the time-step rule.

Every workload is a dict with the mesh, nodal E and h fields [N][S], material
constants, traction patterns [J][N][3], the amplitude table [n_steps][J] and dt.
"""
from __future__ import annotations

import math
import numpy as np

from .mesh import tube_mesh, aneurysm_mesh, tube_for_nodes, plate_mesh, single_triangle, arch_mesh
from .fields import lognormal_fields, gaussian_fields
from .loads import pressure_shear_modes, step_amplitudes, pulsatile_amplitudes, delayed_pressure, ramp

RHO = 1060.0        # kg/m^3 (the paper's 1.06 is read as g/cm^3)
NU = 0.5            # Poisson ratio
KSHEAR = 5.0 / 6.0  # transverse shear factor k
ALPHA = 1.0e3       # mass-proportional damping, 1/s


def inscribed_diameters(xyz: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """Diameter of the circle inscribed in each triangle: 4 A / perimeter."""
    X = xyz[tri]
    a = np.linalg.norm(X[:, 1] - X[:, 0], axis=1)
    b = np.linalg.norm(X[:, 2] - X[:, 1], axis=1)
    c = np.linalg.norm(X[:, 0] - X[:, 2], axis=1)
    area = 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)
    return 4.0 * area / (a + b + c)


def cfl_dt(mesh, E: np.ndarray, rho: float = RHO, safety: float = 0.5) -> float:
    """dt = safety * l_min / c with l_min the smallest inscribed diameter and
    c = sqrt(E_max / rho) the elastic wave speed at the stiffest node and sample."""
    lmin = float(inscribed_diameters(mesh.xyz, mesh.tri).min())
    c = math.sqrt(float(np.max(E)) / rho)
    return safety * lmin / c


def _case(mesh, S, seed, n_steps, load, uniform=False, alpha=ALPHA, dt=None, corr=0.02,
          std=0.1, E_mean=0.7e6, h_mean=1.0e-3, pressure=10.0e3, sample0=0):
    E, h = lognormal_fields(mesh, S, E_mean=E_mean, h_mean=h_mean, corr_length=corr, std=std,
                            seed=seed, uniform=uniform, sample0=sample0)
    if dt is None:
        dt = cfl_dt(mesh, E if S > 0 else np.array([E_mean]))
    if load == "step":
        modes = pressure_shear_modes(mesh)
        amp = step_amplitudes(n_steps, pressure)
    elif load == "pulsatile":
        modes = pressure_shear_modes(mesh, with_shear=True)
        amp = pulsatile_amplitudes(n_steps, dt, with_shear=True)
    else:
        raise ValueError(load)
    return dict(mesh=mesh, S=S, E=E, h=h, rho=RHO, nu=NU, kshear=KSHEAR, alpha=alpha, dt=dt,
                modes=modes, amp=amp, n_steps=n_steps, seed=seed)


def make_case(name: str, S: int | None = None, n_steps: int | None = None, seed: int = 0, **kw):
    """Build a named workload.

    tube_40x40   : R = 1 cm, L = 10 cm, 40 x 40 nodes (1600 nodes, 3120 triangles), S = 8,
                   10 kPa step pressure, damping 1e3 1/s, 0.5 x CFL, 2000 steps.
    aneurysm     : 400 x 500 nodes (200k nodes, 399,200 triangles) with a Gaussian bulge to
                   R = 2 cm, S = 64, pulsatile 10.7 +- 2.7 kPa plus 1 Pa axial shear, ramp 0.2 s.
    aneurysm_50k : the same geometry at 200 x 250 nodes.
    tube_<n>k    : clamped straight tube with about n thousand nodes, step load.
    arch         : synthetic arch with three branches, travelling-wave pressure.
    small tests  : one_triangle, plate, tube_small (12 x 8 nodes).
    cylinder     : the paper's ideal cylinder (Section 3.1): D = 4 cm, L = 30 cm, ends fully
                   fixed, Gaussian marginals E = 0.7 +- 0.07 MPa and h = 4 +- 0.4 mm with
                   correlation length corr (0.95, 3.7 or 7.2 cm), S = 100, mesh level 0 / 1 / 2
                   with 5,074 / 15,136 / 32,994 triangles (level 3: 131,648, near the
                   131,552 of the paper's Table 3); 13 mmHg plus the steady
                   Poiseuille pressure drop and wall shear of 66.59 mL/s (mu = 4 mPa s),
                   ramped in over 5 ms and held.
    """
    if name == "tube_40x40":
        return _case(tube_mesh(40, 40), S or 8, seed, n_steps or 2000, "step", **kw)
    if name == "aneurysm":
        m = aneurysm_mesh(400, 500)
        c = _case(m, S or 64, seed, 1, "pulsatile", **kw)
        steps = n_steps or int(math.ceil(0.8 / c["dt"]))
        c["n_steps"] = steps
        c["amp"] = pulsatile_amplitudes(steps, c["dt"], with_shear=True)
        return c
    if name == "aneurysm_50k":
        m = aneurysm_mesh(200, 250)
        c = _case(m, S or 256, seed, 1, "pulsatile", **kw)
        steps = n_steps or int(math.ceil(0.8 / c["dt"]))
        c["n_steps"] = steps
        c["amp"] = pulsatile_amplitudes(steps, c["dt"], with_shear=True)
        return c
    if name.startswith("tube_") and name.endswith("k"):
        n = int(name[5:-1]) * 1000
        return _case(tube_for_nodes(n), S or 16, seed, n_steps or 1000, "step", **kw)
    if name == "cylinder":
        level = int(kw.pop("level", 2))
        corr = float(kw.pop("corr", 0.037))
        nc, na = [(43, 60), (88, 87), (117, 142), (176, 375)][level]
        R, L = 0.02, 0.30
        m = tube_mesh(nc, na, radius=R, length=L)
        S = 100 if S is None else S
        if kw.pop("host_fields", True):
            E, h = gaussian_fields(m, S, 0.7e6, 0.07e6, 4.0e-3, 0.4e-3, corr, seed)
            E_max = np.max(E)
        else:   # fields drawn elsewhere (e.g. on the device); dt at mean + 6 std
            E, h, E_max = None, None, 0.7e6 + 6 * 0.07e6
        dt = kw.pop("dt", None) or cfl_dt(m, np.array([E_max]))
        n = n_steps or 2000
        mu, Q = 4.0e-3, 66.59e-6
        p0 = 13.0 * 133.322387415                      # 13 mmHg in Pa
        dp = 8.0 * mu * L * Q / (np.pi * R ** 4)       # Poiseuille pressure drop over L
        tau = 4.0 * mu * Q / (np.pi * R ** 3)          # wall shear stress
        zc = m.xyz[m.tri].mean(axis=1)[:, 2]
        modes = pressure_shear_modes(m, delay_modes=[np.ones(m.n_elems), 1.0 - zc / L], with_shear=True)
        r = ramp(dt * np.arange(n), 5.0e-3)
        amp = np.ascontiguousarray(np.stack([r * p0, r * dp, r * tau], axis=1))
        return dict(mesh=m, S=S, E=E, h=h, rho=RHO, nu=NU, kshear=KSHEAR, alpha=kw.pop("alpha", ALPHA),
                    dt=dt, modes=modes, amp=amp, n_steps=n, seed=seed, corr=corr, pressure=p0)
    if name == "tube_small":
        return _case(tube_mesh(12, 8, length=0.03), S or 3, seed, n_steps or 200, "step", **kw)
    if name == "plate":
        m = plate_mesh(6, 5, jitter=0.2, seed=seed)
        m.fixed[[0, 5], :] = 1
        return _case(m, S or 3, seed, n_steps or 50, "step", corr=0.01, **kw)
    if name == "one_triangle":
        m = single_triangle()
        m.fixed[0, :] = 1
        return _case(m, S or 2, seed, n_steps or 20, "step", corr=0.005, **kw)
    if name == "arch":
        m = arch_mesh(**{k: v for k, v in kw.items() if k in ("target_elems",)})
        kw = {k: v for k, v in kw.items() if k not in ("target_elems",)}
        c = _case(m, S or 256, seed, 1, "step", **kw)
        # path length from the inlet: arch nodes by ring, branch nodes by their base
        s_node = _arch_path_length(m)
        steps = n_steps or int(math.ceil(0.8 / c["dt"]))
        modes, amp = delayed_pressure(m, s_node, steps, c["dt"])
        c.update(modes=modes, amp=amp, n_steps=steps)
        return c
    raise ValueError(f"unknown case {name}")


def with_dt(name: str, case: dict, dt: float) -> dict:
    """The workload `name` with time step dt: the shards of one ensemble drawn on several
    processes agree on the step of its stiffest realisation. The load table is rebuilt
    where it depends on dt (the pulsatile and travelling-wave loads)."""
    c = dict(case, dt=float(dt))
    if name in ("aneurysm", "aneurysm_50k"):
        c["amp"] = pulsatile_amplitudes(c["n_steps"], c["dt"], with_shear=True)
    elif name == "arch":
        c["modes"], c["amp"] = delayed_pressure(c["mesh"], _arch_path_length(c["mesh"]), c["n_steps"], c["dt"])
    return c


def _arch_path_length(m) -> np.ndarray:
    nc, na = m.meta["nc"], m.meta["na"]
    s = m.meta["s"]
    cen = m.meta["centreline"]
    out = np.empty(m.n_nodes)
    out[: nc * na] = np.repeat(s, nc)
    rest = np.arange(nc * na, m.n_nodes)
    if rest.size:
        p = m.xyz[rest]
        d = np.linalg.norm(p[:, None, :] - cen[None, :, :], axis=2)
        k = np.argmin(d, axis=1)
        out[rest] = s[k] + d[np.arange(rest.size), k]
    return out
