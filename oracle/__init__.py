"""FP64 CPU oracle for the explicit ensemble update of the 3-dof wall shell.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline arm are the only callers. The CUDA library never imports or links this
package and shares no code with it.

The numerical core is plain C (ens_oracle.c, compiled with gcc + OpenMP into
oracle/_build/liboracle.so by build()). Arrays cross the boundary sample-outermost
([S][N][3]); the helpers here convert from and to the synthetic-input layout
([N][S] fields) only by transposition.

Sections followed (paper: Li & Schiavazzi, arXiv 2101.09059):
  element_matrices     Section 2.2.1 (B, C, k_e)
  gauss_eh, lumped_mass Section 2.2.1 three-point rule; Section 2.3 lumped M~
  internal_force       Section 2.4 assembly-free element products
  run                  Section 2.3 Eq. (dynamicsCD), C = alpha M, Taylor start (reading)
  stats                ensemble mean and sample variance (Section 3.1 ensemble bands)
Pinned by tests/test_oracle_*.py; see the module docstrings there for each pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ens_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only) if the library is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.orc_element_matrix.argtypes = [_dp, f64, f64, _dp, _dp]
        L.orc_element_matrix.restype = ctypes.c_int
        L.orc_element_matrices.argtypes = [i32, _dp, _ip, f64, f64, _dp, _dp]
        L.orc_element_matrices.restype = ctypes.c_int
        L.orc_gauss_eh.argtypes = [i32, i32, i32, _ip, _dp, _dp, _dp, _dp]
        L.orc_gauss_eh.restype = None
        L.orc_lumped_mass.argtypes = [i32, i32, i32, _ip, _dp, _dp, f64, _dp]
        L.orc_lumped_mass.restype = None
        L.orc_internal_force.argtypes = [i32, i32, i32, _ip, _dp, _dp, _dp, _dp]
        L.orc_internal_force.restype = None
        L.orc_cd_start.argtypes = [i32, i32, i32, _ip, _dp, _dp, _dp, f64, f64, _u8p, i32, _dp,
                                   _dp, _dp, _dp, _dp]
        L.orc_cd_start.restype = None
        L.orc_cd_steps.argtypes = [i32, i32, i32, _ip, _dp, _dp, _dp, f64, f64, _u8p, i32, _dp,
                                   i64, _dp, i64, i64, _dp, _dp]
        L.orc_cd_steps.restype = ctypes.c_int
        L.orc_stats.argtypes = [i32, i64, _dp, _dp, _dp]
        L.orc_stats.restype = None
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_ip)
    if a.dtype == np.uint8:
        return a.ctypes.data_as(_u8p)
    raise TypeError(a.dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def element_matrix(X, nu: float, kshear: float):
    """Global-frame element stiffness per unit (E h) of one triangle X [3][3] -> ([9][9], area)."""
    X = _c(X, np.float64).reshape(9)
    K = np.zeros(81)
    A = np.zeros(1)
    rc = lib().orc_element_matrix(_p(X), nu, kshear, _p(K), _p(A))
    if rc != 0:
        raise ValueError("degenerate triangle")
    return K.reshape(9, 9), float(A[0])


def element_matrices(xyz, tri, nu: float, kshear: float):
    """[E][9][9] global element matrices per unit (E h) and [E] areas."""
    xyz = _c(xyz, np.float64)
    tri = _c(tri, np.int32)
    E = tri.shape[0]
    K = np.zeros((E, 81))
    A = np.zeros(E)
    rc = lib().orc_element_matrices(E, _p(xyz), _p(tri), nu, kshear, _p(K), _p(A))
    if rc != 0:
        raise ValueError(f"degenerate triangle {-rc - 1}")
    return K.reshape(E, 9, 9), A


def gauss_eh(tri, E_node, h_node):
    """E_node, h_node: [N][S] -> (eh, hbar) each [E][S] (three-point Gauss products)."""
    tri = _c(tri, np.int32)
    N, S = E_node.shape
    En = _c(np.asarray(E_node).T, np.float64)
    hn = _c(np.asarray(h_node).T, np.float64)
    E = tri.shape[0]
    eh = np.zeros((S, E))
    hb = np.zeros((S, E))
    lib().orc_gauss_eh(N, E, S, _p(tri), _p(En), _p(hn), _p(eh), _p(hb))
    return eh.T.copy(), hb.T.copy()


def lumped_mass(n_nodes: int, tri, area, hbar, rho: float):
    """hbar [E][S] -> m [N][S]."""
    tri = _c(tri, np.int32)
    E, S = hbar.shape
    hb = _c(np.asarray(hbar).T, np.float64)
    m = np.zeros((S, n_nodes))
    lib().orc_lumped_mass(n_nodes, E, S, _p(tri), _p(_c(area, np.float64)), _p(hb), rho, _p(m))
    return m.T.copy()


class Model:
    """Element matrices, Gauss products and lumped masses of one workload (all FP64)."""

    def __init__(self, case, samples=None, coeffs=None):
        """coeffs = (eh [E][S], rho_hbar [E][S]): per-element coefficients given directly
        (the Gauss products and rho times the element-mean thickness) instead of the
        nodal fields case["E"], case["h"]."""
        mesh = case["mesh"]
        self.case = case
        self.N = mesh.n_nodes
        self.E = mesh.n_elems
        self.tri = _c(mesh.tri, np.int32)
        self.fixed = _c(mesh.fixed, np.uint8).reshape(-1)
        self.Kg, self.area = element_matrices(mesh.xyz, mesh.tri, case["nu"], case["kshear"])
        self.Kg = _c(self.Kg.reshape(self.E, 81), np.float64)
        if coeffs is None:
            E_node = case["E"] if samples is None else case["E"][:, samples]
            h_node = case["h"] if samples is None else case["h"][:, samples]
            eh, hb = gauss_eh(mesh.tri, E_node, h_node)
            rho = case["rho"]
        else:
            eh, hb = (np.asarray(a, dtype=np.float64) for a in coeffs)
            if samples is not None:
                eh, hb = eh[:, samples], hb[:, samples]
            rho = 1.0                               # hb already carries rho
        self.S = eh.shape[1]
        self.eh_se = _c(eh.T, np.float64)          # [S][E]
        self.hbar_se = _c(hb.T, np.float64)
        m = lumped_mass(self.N, mesh.tri, self.area, hb, rho)
        self.m_sn = _c(m.T, np.float64)            # [S][N]
        self.alpha = float(case["alpha"])
        self.dt = float(case["dt"])
        self.modes = _c(case["modes"], np.float64)
        self.J = int(self.modes.shape[0])
        self.amp = _c(case["amp"], np.float64)

    def internal_force(self, u_sn3):
        """u [S][N][3] -> K_s u_s [S][N][3]."""
        u = _c(u_sn3, np.float64)
        f = np.zeros_like(u)
        lib().orc_internal_force(self.N, self.E, self.S, _p(self.tri), _p(self.Kg), _p(self.eh_se),
                                 _p(u), _p(f))
        return f

    def start(self, u0=None, v0=None):
        """Return (u_{-1}, u_0) for the initial state (rest by default)."""
        shape = (self.S, self.N, 3)
        u0 = np.zeros(shape) if u0 is None else _c(u0, np.float64)
        v0 = np.zeros(shape) if v0 is None else _c(v0, np.float64)
        up = np.zeros(shape)
        lib().orc_cd_start(self.N, self.E, self.S, _p(self.tri), _p(self.Kg), _p(self.eh_se),
                           _p(self.m_sn), self.alpha, self.dt, _p(self.fixed), self.J,
                           _p(self.modes), _p(self.amp[0].copy()), _p(u0), _p(v0), _p(up))
        u0 = u0.copy()
        u0.reshape(self.S, -1)[:, self.fixed.astype(bool)] = 0.0
        return up, u0

    def steps(self, u_prev, u_cur, step0: int, n: int):
        """Advance (u_prev, u_cur) in place by n steps of Eq. (dynamicsCD) from step index step0."""
        assert u_prev.dtype == np.float64 and u_prev.flags.c_contiguous
        assert u_cur.dtype == np.float64 and u_cur.flags.c_contiguous
        rc = lib().orc_cd_steps(self.N, self.E, self.S, _p(self.tri), _p(self.Kg), _p(self.eh_se),
                                _p(self.m_sn), self.alpha, self.dt, _p(self.fixed), self.J,
                                _p(self.modes), self.amp.shape[0], _p(self.amp), step0, n,
                                _p(u_prev), _p(u_cur))
        if rc != 0:
            raise ValueError("load table too short")
        return u_prev, u_cur

    def run(self, n: int):
        """u_n [S][N][3] after n steps from rest, plus u_{n-1}."""
        up, uc = self.start()
        self.steps(up, uc, 0, n)
        return uc, up


def stats(u_sk):
    """u [S][K] -> (mean [K], sample variance [K]) by the two-pass formula."""
    u = _c(u_sk, np.float64)
    S = u.shape[0]
    K = int(np.prod(u.shape[1:]))
    mean = np.zeros(K)
    var = np.zeros(K)
    lib().orc_stats(S, K, _p(u), _p(mean), _p(var))
    return mean.reshape(u.shape[1:]), var.reshape(u.shape[1:])
