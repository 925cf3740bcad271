"""The allocation-free internal force (ens_internal_force_noalloc) through the C ABI.

Some callers of this library may not allocate device memory when they need a force
evaluation: a host framework that owns every device allocation, or a time loop in which
cudaMalloc (and the device synchronisation it can imply) is not allowed. For them the
library stages through one static device array instead. This test checks that entry
point against the allocating ens_internal_force on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next result), and that a
context too large for the array is refused. The file sorts last so that a run stopping at
its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2101_09059_gb300 as ens  # noqa: E402
from paper_2101_09059_gb300 import _lib  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _call_noalloc(e, u_ncs):
    L = _lib.load()
    u_d = torch.from_numpy(np.ascontiguousarray(u_ncs)).cuda()
    f_d = torch.full_like(u_d, np.nan)
    rc = L.ens_internal_force_noalloc(e._ctx, ctypes.c_void_p(u_d.data_ptr()),
                                      ctypes.c_void_p(f_d.data_ptr()))
    assert rc == 0, L.ens_last_error(e._ctx).decode()
    e.stream.synchronize()
    return f_d.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "kahan32", "fp32_force"])
@pytest.mark.parametrize("name,S", [("tube_small", 5), ("tube_40x40", 8)])
def test_noalloc_matches_allocating_entry_point(name, S, precision):
    case = synth.make_case(name, S=S)
    e = ens.Ensemble.from_case(case, precision=precision)
    rng = np.random.default_rng(11)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for call in range(2):
        u = 1e-3 * rng.standard_normal((e.N, 3, e.S))
        f_ref = e.internal_force(u)
        f = _call_noalloc(e, u)
        assert np.isfinite(f).all()
        err = np.linalg.norm(f - f_ref) / np.linalg.norm(f_ref)
        assert err <= tol, (call, err)
    e.close()


def test_noalloc_rejects_context_above_the_static_size():
    case = synth.make_case("tube_20k", S=64, n_steps=4)
    e = ens.Ensemble.from_case(case, precision="fp64")   # 20k x 3 x 64 x 16 B > 32 MiB
    L = _lib.load()
    u_d = torch.zeros((e.N, 3, e.S), dtype=torch.float64, device="cuda")
    f_d = torch.zeros_like(u_d)
    rc = L.ens_internal_force_noalloc(e._ctx, ctypes.c_void_p(u_d.data_ptr()),
                                      ctypes.c_void_p(f_d.data_ptr()))
    assert rc == -1
    assert "static scratch" in L.ens_last_error(e._ctx).decode()
    e.close()
