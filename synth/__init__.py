"""Seeded synthetic inputs for the ensemble wall solver.

This package generates the *inputs* of the explicit ensemble update: surface meshes,
fixed-dof masks, nodal random fields for the elastic modulus E and the thickness h,
nodal traction modes with their amplitude tables, and the time step rule. It holds
none of the update's own arithmetic (no element matrix, no Gauss rule, no lumped
mass, no time stepping, no statistics): both the CUDA library and the FP64 oracle
consume the arrays produced here, and neither is imported by this package.

All units are SI (m, Pa, kg/m^3, s).
"""
from .mesh import Mesh, tube_mesh, aneurysm_mesh, tube_for_nodes, plate_mesh, single_triangle, arch_mesh
from .fields import gmrf_fields, lognormal_fields, matern_correlation
from .loads import pressure_shear_modes, step_amplitudes, pulsatile_amplitudes, waveform, peak_amplitudes
from .kl import kl_basis, kl_coefficients, kl_fields
from .configs import cfl_dt, make_case

__all__ = [
    "Mesh", "tube_mesh", "aneurysm_mesh", "tube_for_nodes", "plate_mesh", "single_triangle", "arch_mesh",
    "gmrf_fields", "lognormal_fields", "matern_correlation",
    "pressure_shear_modes", "step_amplitudes", "pulsatile_amplitudes", "waveform", "peak_amplitudes",
    "kl_basis", "kl_coefficients", "kl_fields",
    "cfl_dt", "make_case",
]
