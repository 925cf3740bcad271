"""Output statistics on the device (ens_quantity_*, ens_row_stats_device, probes) against
the FP64 oracle (oracle/outputs.py) on the oracle's own trajectory.

Tolerances: the row statistics of the same input rows are compared bit for bit for the
quantiles (both sides sort and evaluate x_j + g (x_{j+1} - x_j) without fused operations)
and to 1e-14 relative for mean and variance (summation order differs). Quantities of a
state reached by stepping inherit the trajectory tolerance (1e-10 relative for the FP64
form, 1e-5 for the binary32 forms); stress is a fixed linear map of u scaled by E, so the
same relative bound holds row-wise against the largest row value."""
import numpy as np
import pytest

import oracle
import oracle.outputs as oo
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_09059_gb300 as ens  # noqa: E402
from paper_2101_09059_gb300.ensemble import (QTY_DISPLACEMENT, QTY_DISP_MAGNITUDE, QTY_STRESS,  # noqa: E402
                                             row_stats_device)

Q = [0.0, 0.05, 0.25, 0.5, 0.75, 0.95, 1.0, 0.123]
TOL = {"fp64": 1e-10, "fp32_force": 1e-5, "kahan32": 1e-5}


def _axis(m):
    z = m.xyz[:, 2]
    return np.array([[0.0, 0.0, z.min() - 0.01], [0.0, 0.0, z.max() + 0.01]])


@pytest.mark.parametrize("S", [1, 2, 7, 64, 200])
def test_row_stats_bitwise_quantiles(S):
    rng = np.random.Generator(np.random.Philox(key=S))
    rows = rng.standard_normal((333, S)) * 1e-4
    rows[5] = 3.0            # a constant row
    rows[6, : S // 2] = 0.0  # ties
    m, v, q = row_stats_device(torch.from_numpy(rows).cuda(), Q)
    mo, vo, qo = oo.row_stats(rows, Q)
    assert np.array_equal(q.cpu().numpy(), qo)
    assert np.allclose(m.cpu().numpy(), mo, rtol=1e-14, atol=1e-14 * np.abs(rows).max())
    assert np.allclose(v.cpu().numpy(), vo, rtol=1e-13, atol=1e-28)


def _run_both(name, S, n, precision="fp64", **kw):
    case = synth.make_case(name, S=S, n_steps=n + 10, seed=3, **kw)
    e = ens.Ensemble.from_case(case, precision=precision)
    e.set_centerline(_axis(case["mesh"]))
    e.step(n)
    u_or = oracle.Model(case).run(n)[0]        # [S][N][3]
    return case, e, u_or


@pytest.mark.parametrize("precision", ["fp64", "fp32_force", "kahan32"])
def test_quantities_match_oracle(precision):
    case, e, u_or = _run_both("tube_40x40", 8, 300, precision)
    m = case["mesh"]
    tol = TOL[precision]
    rows_or = {QTY_DISPLACEMENT: oo.displacement_rows(u_or), QTY_DISP_MAGNITUDE: oo.magnitude_rows(u_or),
               QTY_STRESS: oo.element_stress(m.xyz, m.tri, u_or, case["E"], case["nu"], case["kshear"], _axis(m))}
    for qty, ref in rows_or.items():
        got = e.quantity_device(qty).cpu().numpy()
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), qty
        mean, var, quant = e.quantity_stats(qty, Q)
        mo, vo, qo = oo.row_stats(ref, Q)
        assert np.abs(mean - mo).max() <= tol * np.abs(ref).max(), qty
        assert np.abs(quant - qo).max() <= tol * np.abs(ref).max(), qty
        assert np.abs(np.sqrt(var) - np.sqrt(vo)).max() <= tol * np.abs(ref).max() * 2, qty
    e.close()


def test_stress_of_the_pressurised_tube_is_hoop_dominated():
    """A settled step-pressure state: mean hoop stress mid-tube near p R / h, shears small."""
    case, e, _ = _run_both("tube_40x40", 4, 1500)
    mean, _, _ = e.quantity_stats(QTY_STRESS)
    s = mean.reshape(-1, 6)
    m = case["mesh"]
    zc = m.xyz[m.tri].mean(axis=1)[:, 2]
    mid = np.abs(zc - 0.05) < 0.01
    p, R, h = 1e4, 0.01, 1e-3
    assert 0.6 * p * R / h < s[mid, 1].mean() < 1.4 * p * R / h
    assert np.abs(s[mid][:, [3, 4, 5]]).max() < 0.2 * s[mid, 1].mean()
    e.close()


def test_probes_record_the_trajectory():
    case = synth.make_case("tube_40x40", S=5, n_steps=400, seed=4)
    m = case["mesh"]
    e = ens.Ensemble.from_case(case, precision="fp64")
    e.set_centerline(_axis(m))
    nodes, elems = [17, 800, 1599], [0, 1500, 3119]
    e.set_probes(nodes, elems, stride=64, capacity=4)
    e.step(100)
    e.step(250)                       # records at 64, 128, 192, 256; 320 is past capacity
    steps, u, sig = e.probes()
    assert steps.tolist() == [64, 128, 192, 256]
    mod = oracle.Model(case)
    up, uc = mod.start()
    done = 0
    for k, st in enumerate(steps):
        mod.steps(up, uc, done, int(st) - done)
        done = int(st)
        ref_u = np.transpose(uc[:, nodes, :], (1, 2, 0))
        assert np.abs(u[k] - ref_u).max() <= 1e-10 * np.abs(uc).max()
        ref_s = oo.element_stress(m.xyz, m.tri, uc, case["E"], case["nu"], case["kshear"], _axis(m))
        ref_s = ref_s.reshape(-1, 6, 5)[elems]
        assert np.abs(sig[k] - ref_s).max() <= 1e-10 * np.abs(ref_s).max() + 1e-300
    e.reset()
    assert e.probes()[0].size == 0
    e.set_probes(stride=0)
    e.step(128)
    assert e.probes()[0].size == 0
    e.close()


def test_output_errors():
    case = synth.make_case("tube_small", S=3)
    e = ens.Ensemble.from_case(case, precision="fp64")
    with pytest.raises(ens.EnsError) as x:
        e.quantity_device(QTY_STRESS)          # no centreline yet
    assert x.value.code == -8
    with pytest.raises(ens.EnsError):
        e.quantity_stats(QTY_DISPLACEMENT, [1.5])
    with pytest.raises(ens.EnsError):
        e.set_probes([10_000], stride=4, capacity=2)
    with pytest.raises(ens.EnsError):
        e.set_probes([], [0], stride=4, capacity=2)   # element probes need a centreline
    e.close()
    plate = synth.make_case("plate", S=2)
    e = ens.Ensemble.from_case(plate, precision="fp64")
    with pytest.raises(ens.EnsError) as x:   # every wall normal (+z) parallel to the axis
        e.set_centerline(np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]]))
    assert x.value.code == -1
    e.close()


def test_full_size_aneurysm_outputs_sampled():
    """The 200k-node aneurysm at S = 64 (FP32-force, the launch shape the benchmark uses):
    stress and |u| rows of two samples against the oracle after 120 steps."""
    case = synth.make_case("aneurysm", S=64, n_steps=130, seed=0)
    m = case["mesh"]
    e = ens.Ensemble.from_case(case, precision="fp32_force")
    e.set_centerline(_axis(m))
    e.step(120)
    pick = [0, 63]
    u_or = oracle.Model(case, samples=pick).run(120)[0]
    got = e.quantity_device(QTY_STRESS).cpu().numpy()[:, pick]
    ref = oo.element_stress(m.xyz, m.tri, u_or, case["E"][:, pick], case["nu"], case["kshear"], _axis(m))
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    mag = e.quantity_device(QTY_DISP_MAGNITUDE).cpu().numpy()[:, pick]
    assert np.abs(mag - oo.magnitude_rows(u_or)).max() <= 1e-5 * np.abs(mag).max()
    mean, var, quant = e.quantity_stats(QTY_DISP_MAGNITUDE, [0.05, 0.5, 0.95])
    assert np.all(quant[:, 0] <= quant[:, 1]) and np.all(quant[:, 1] <= quant[:, 2])
    e.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_force", "kahan32"])
@pytest.mark.parametrize("stride", [1, 7])
def test_running_peak_matches_oracle(precision, stride):
    """The running peak of |u| per node and realisation (ens_set_peak) over 2000 steps of
    the 40 x 40 tube against oracle.outputs.peak_magnitude on the same recorded steps,
    within the trajectory tolerance of the form, relative to the largest peak; its row
    statistics against the oracle's; graph replays and direct launches give the same
    peak bit for bit; ens_reset clears it."""
    from paper_2101_09059_gb300.ensemble import FLAG_NO_GRAPH, QTY_PEAK_MAGNITUDE
    case = synth.make_case("tube_40x40", S=8, seed=5)
    n = case["n_steps"]
    ref, _, u_end = oo.peak_magnitude(oracle.Model(case), n, stride)
    peaks = []
    for flags in (0, FLAG_NO_GRAPH):
        e = ens.Ensemble.from_case(case, precision=precision, flags=flags)
        with pytest.raises(ens.EnsError) as ei:
            e.quantity_device(QTY_PEAK_MAGNITUDE)
        assert ei.value.code == -8
        e.set_peak(stride)
        for part in (1, 700, 299, n - 1000):
            e.step(part)
        p = e.quantity_device(QTY_PEAK_MAGNITUDE).cpu().numpy()
        peaks.append(p)
        err = np.abs(p - ref).max() / np.abs(ref).max()
        print(f"peak {precision} stride {stride}: max rel {err:.2e}")
        assert err < TOL[precision]
        u = e.displacement()
        assert np.linalg.norm(u - u_end) <= TOL[precision] * np.linalg.norm(u_end)
        m, v, q = e.quantity_stats(QTY_PEAK_MAGNITUDE, Q)
        mo, vo, qo = oo.row_stats(ref, Q)
        assert np.abs(q - qo).max() <= TOL[precision] * np.abs(ref).max()
        assert np.abs(m - mo).max() <= TOL[precision] * np.abs(ref).max()
        e.reset()
        assert not e.quantity_device(QTY_PEAK_MAGNITUDE).cpu().numpy().any()
        e.close()
    assert np.array_equal(peaks[0], peaks[1])


def test_running_peak_members_cannot_join_a_batch():
    case = synth.make_case("tube_small", S=4, n_steps=20)
    a = ens.Ensemble.from_case(case, precision="kahan32")
    b = ens.Ensemble.from_case(case, precision="kahan32")
    a.set_peak(1)
    with pytest.raises(ens.EnsError) as ei:
        ens.Batch([a, b])
    assert ei.value.code == -8
    a.close()
    b.close()


def test_full_size_aneurysm_running_peak_sampled():
    """The 200k-node aneurysm at S = 64, FP32-force, peak recorded every 10 steps over 1000
    steps: two realisations against the oracle's peak (realisations are independent, so the
    subset is exact), within the form's trajectory tolerance."""
    from paper_2101_09059_gb300.ensemble import QTY_PEAK_MAGNITUDE
    case = synth.make_case("aneurysm", S=64, n_steps=1000, seed=0)
    e = ens.Ensemble.from_case(case, precision="fp32_force")
    e.set_peak(10)
    e.step(1000)
    p = e.quantity_device(QTY_PEAK_MAGNITUDE).cpu().numpy()
    e.close()
    picks = [5, 50]
    ref, _, _ = oo.peak_magnitude(oracle.Model(case, samples=picks), 1000, 10)
    for k, s in enumerate(picks):
        err = np.abs(p[:, s] - ref[:, k]).max() / np.abs(ref[:, k]).max()
        print(f"aneurysm peak sample {s}: max rel {err:.2e}")
        assert err < TOL["fp32_force"]
