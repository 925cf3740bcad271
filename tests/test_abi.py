"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a,
loads, exports every function include/ens.h declares, and rejects invalid arguments
before touching the device."""
import ctypes

import numpy as np
import pytest

import paper_2101_09059_gb300 as ens
from paper_2101_09059_gb300 import _lib


@pytest.fixture(scope="module")
def L():
    return _lib.load()


def test_every_declared_symbol_is_exported(L):
    names = _lib.declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(L):
    for code in range(0, -9, -1):
        s = L.ens_error_string(code).decode()
        assert s and s != "unknown status"
    assert L.ens_error_string(-99).decode() == "unknown status"
    assert L.ens_last_error(None).decode() == ""


def _args(N=3, E=1, S=2):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=np.float64)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    En = np.full((N, S), 1e6)
    hn = np.full((N, S), 1e-3)
    return xyz, tri, En, hn


def _create(L, xyz, tri, En, hn, S, **kw):
    p = dict(rho=1000.0, nu=0.3, kshear=5 / 6, alpha=0.0, dt=1e-7, precision=0, flags=0)
    p.update(kw)
    mesh = _lib.ens_mesh(xyz.shape[0], tri.shape[0], xyz.ctypes.data, tri.ctypes.data, None)
    params = _lib.ens_params(p["rho"], p["nu"], p["kshear"], p["alpha"], p["dt"], p["precision"],
                             p["flags"])
    out = ctypes.c_void_p(1234)
    rc = L.ens_create(ctypes.byref(mesh), S, ctypes.c_void_p(En.ctypes.data),
                      ctypes.c_void_p(hn.ctypes.data), ctypes.byref(params), None, None,
                      ctypes.byref(out))
    return rc, out


@pytest.mark.parametrize("bad", [
    dict(nu=1.0), dict(nu=-0.1), dict(rho=0.0), dict(dt=0.0), dict(dt=float("nan")),
    dict(alpha=-1.0), dict(kshear=0.0), dict(precision=3), dict(flags=8), dict(flags=1 << 12),
    dict(flags=16 | 32),
])
def test_create_rejects_bad_parameters(L, bad):
    xyz, tri, En, hn = _args()
    rc, out = _create(L, xyz, tri, En, hn, 2, **bad)
    assert rc == -1 and not out.value


def test_create_rejects_bad_fields_and_mesh(L):
    xyz, tri, En, hn = _args()
    En2 = En.copy()
    En2[1, 0] = -1.0
    assert _create(L, xyz, tri, En2, hn, 2)[0] == -1
    hn2 = hn.copy()
    hn2[0, 1] = np.inf
    assert _create(L, xyz, tri, En, hn2, 2)[0] == -1
    assert _create(L, xyz, tri, En, hn, 0)[0] == -1
    xyz2 = xyz.copy()
    xyz2[0, 0] = np.nan
    assert _create(L, xyz2, tri, En, hn, 2)[0] == -1


def test_null_arguments(L):
    assert L.ens_create(None, 1, None, None, None, None, None, None) == -1
    assert L.ens_step(None, 1) == -1
    assert L.ens_stats(None, None, None) == -1
    assert L.ens_info(None, None) == -1
    L.ens_destroy(None)


def test_python_binding_has_no_cpu_path():
    # The binding only marshals arguments: every compute method goes through the ABI.
    import inspect
    src = inspect.getsource(ens.ensemble)
    assert "oracle" not in src and "import synth" not in src


@pytest.mark.parametrize("case", ["kappa0", "kappa_nan", "node_out_of_range", "orphan_node",
                                  "zero_area", "no_out"])
def test_field_sampler_create_rejects_bad_input(L, case):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.float64)
    tri = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    corr = 0.02
    if case == "kappa0":
        corr = 0.0
    elif case == "kappa_nan":
        corr = float("nan")
    elif case == "node_out_of_range":
        tri = np.array([[0, 1, 2], [1, 4, 2]], dtype=np.int32)
    elif case == "orphan_node":
        tri = np.array([[0, 1, 2]], dtype=np.int32)
    elif case == "zero_area":
        xyz[3] = [2, 0, 0]
        tri = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    out = ctypes.c_void_p(1234)
    rc = L.gmrf_create(xyz.shape[0], tri.shape[0], ctypes.c_void_p(xyz.ctypes.data),
                       ctypes.c_void_p(tri.ctypes.data), corr, None,
                       None if case == "no_out" else ctypes.byref(out))
    assert rc == -1
    assert L.gmrf_last_error(None).decode()
    if case != "no_out":
        assert out.value is None


@pytest.mark.parametrize("case", ["S0", "S_big", "nq_big", "q_range", "q_nan", "rows_null", "quant_null"])
def test_row_stats_rejects_bad_arguments_before_device_work(L, case):
    n_rows, S, n_q = 4, 8, 2
    q = np.array([0.05, 0.95])
    rows = ctypes.c_void_p(0x1000)       # never dereferenced: the checks come first
    quant = ctypes.c_void_p(0x2000)
    if case == "S0":
        S = 0
    elif case == "S_big":
        S = 16385
    elif case == "nq_big":
        n_q, q = 1025, np.full(1025, 0.5)
    elif case == "q_range":
        q = np.array([0.05, 1.5])
    elif case == "q_nan":
        q = np.array([float("nan"), 0.5])
    elif case == "rows_null":
        rows = None
    elif case == "quant_null":
        quant = None
    rc = L.ens_row_stats_device(n_rows, S, rows, n_q, ctypes.c_void_p(q.ctypes.data), None, None, quant, None)
    assert rc == -1
