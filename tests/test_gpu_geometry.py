"""Geometry update with selective stiffness re-assembly on the device
(ens_set_geometry_update, Section 2.3) against the oracle (oracle/geometry.py).

Tolerances: the trajectory tolerances of the linear method (1e-10 relative L2 for the
FP64 form, 1e-5 for the binary32 forms). The re-assembly evaluates the element frame and
coupling blocks with the set-up kernel's arithmetic on the deformed coordinates, and the
per-realisation step applies them in the linear kernel's operation order, so a run that
never re-assembles is the linear run bit for bit."""
import numpy as np
import pytest

import synth
from oracle import geometry as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_09059_gb300 as ens  # noqa: E402
from paper_2101_09059_gb300.ensemble import FLAG_NO_GRAPH  # noqa: E402

TOL = {"fp64": 1e-10, "fp32_force": 1e-5, "kahan32": 1e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case():
    """The 40 x 40 tube of the configuration (10 kPa step, S = 8)."""
    return synth.make_case("tube_40x40", S=8, seed=2)


@pytest.mark.parametrize("precision", ["fp64", "fp32_force", "kahan32"])
def test_without_reassembly_the_run_is_the_linear_run_bitwise(precision):
    case = _case()
    lin = ens.Ensemble.from_case(case, precision=precision)
    lin.step(300)
    geo = ens.Ensemble.from_case(case, precision=precision)
    geo.set_geometry_update(100000)
    geo.step(300)
    assert np.array_equal(geo.displacement(), lin.displacement())
    lin.close()
    geo.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_force", "kahan32"])
def test_geometry_update_matches_oracle(precision):
    case = _case()
    n, k = case["n_steps"], 10
    ref = og.run_updated(case, n, k)
    e = ens.Ensemble.from_case(case, precision=precision)
    e.set_geometry_update(k)
    for part in (1, 733, 266, n - 1000):
        e.step(part)
    u = e.displacement()
    err = _rel(u, ref)
    print(f"geometry update {precision}, k = {k}: rel-L2 {err:.3e}")
    assert err < TOL[precision]
    # the update changes the response by far more than the tolerance
    lin = ens.Ensemble.from_case(case, precision=precision)
    lin.step(n)
    assert _rel(lin.displacement(), ref) > 1e-3
    # reset re-assembles on the reference surface: the rerun is identical
    e.reset()
    e.step(n)
    assert np.array_equal(e.displacement(), u)
    e.set_geometry_update(0)            # back to the linear method
    e.reset()
    e.step(n)
    assert np.array_equal(e.displacement(), lin.displacement())
    e.close()
    lin.close()


def test_geometry_update_members_cannot_join_a_batch():
    case = synth.make_case("tube_small", S=4, n_steps=20)
    a = ens.Ensemble.from_case(case, precision="kahan32")
    b = ens.Ensemble.from_case(case, precision="kahan32")
    a.set_geometry_update(5)
    with pytest.raises(ens.EnsError) as ei:
        ens.Batch([a, b])
    assert ei.value.code == -8
    a.close()
    b.close()


def test_geometry_update_on_the_paper_cylinder_sampled():
    """The paper's cylinder (Section 3.1) at its finest Table-2 mesh (32,994 triangles),
    S = 100, compensated form, re-assembly every 50 steps over 1000 steps: two realisations
    against the oracle."""
    case = synth.make_case("cylinder", level=2, S=100, n_steps=1000)
    e = ens.Ensemble.from_case(case, precision="kahan32")
    e.set_geometry_update(50)
    e.step(1000)
    u = e.displacement()
    e.close()
    picks = [7, 93]
    ref = og.run_updated(case, 1000, 50, samples=picks)
    for k, s in enumerate(picks):
        err = _rel(u[s], ref[k])
        print(f"cylinder geometry update sample {s}: rel-L2 {err:.2e}")
        assert err < TOL["kahan32"]


@pytest.mark.parametrize("precision", ["fp64", "kahan32"])
def test_geometry_update_graph_replays_equal_direct_launches(precision):
    """Re-assembly every 80 steps: each segment replays captured 32-step graphs, and the
    segments alternate between the two per-realisation block buffers (two kept graphs).
    The run equals the one launched step by step, bit for bit, and so do the runs after
    a reset, after the peak tracking adds a launch, and after the update is switched off."""
    case = _case()
    runs = []
    for flags in (0, FLAG_NO_GRAPH):
        e = ens.Ensemble.from_case(case, precision=precision, flags=flags)
        e.set_geometry_update(80)
        e.step(400)
        u = [e.displacement()]
        e.reset()
        e.set_peak(1)
        e.step(330)
        u.append(e.displacement())
        e.set_geometry_update(0)
        e.step(130)
        u.append(e.displacement())
        runs.append(u)
        e.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32_force", "kahan32"])
def test_geometry_update_with_a_ragged_sample_count(precision):
    """S = 5: the per-realisation blocks and the correction carry padded sample lanes
    (Sp = 8), which must neither feed the real samples nor turn non-finite; re-assembly
    every 25 steps over 600 steps against the oracle at the form's tolerance."""
    case = synth.make_case("tube_40x40", S=5, seed=4, n_steps=600)
    ref = og.run_updated(case, 600, 25)
    e = ens.Ensemble.from_case(case, precision=precision)
    e.set_geometry_update(25)
    e.step(600)
    u = e.displacement()
    e.close()
    assert u.shape == ref.shape and np.all(np.isfinite(u))
    err = _rel(u, ref)
    print(f"ragged geometry update {precision}: rel-L2 {err:.3e}")
    assert err < TOL[precision]
