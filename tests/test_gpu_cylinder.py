"""The paper's ideal cylinder (Section 3.1; workload "cylinder"): D = 4 cm, L = 30 cm,
ends fully fixed, Gaussian Matérn fields for E and h, 13 mmHg plus the steady Poiseuille
load, run to steady state on the device with S = 100 realisations.

Section 3.1 reports, one diameter away from the fixed ends, a mean displacement consistent
with the homogeneous solution at the mean E and h, and a 5 %-95 % band that widens as the
correlation length grows (0.95, 3.7, 7.2 cm). Both are checked here on the device's
output statistics, and two realisations of the coarse mesh against the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_09059_gb300 as ens  # noqa: E402
from paper_2101_09059_gb300.ensemble import QTY_DISP_MAGNITUDE  # noqa: E402

STEADY = 0.02   # s: 5 ms ramp, then > 7 damping times (2 / alpha = 2 ms)


def _steady(corr, level=1, S=100, precision="fp32_force"):
    case = synth.make_case("cylinder", level=level, corr=corr, S=S, n_steps=1, seed=11)
    n = int(np.ceil(STEADY / case["dt"]))
    case = synth.make_case("cylinder", level=level, corr=corr, S=S, n_steps=n + 1, seed=11)
    e = ens.Ensemble.from_case(case, precision=precision)
    e.step(n)
    return case, e


def test_mean_displacement_matches_the_homogeneous_solution_and_bands_widen():
    widths = []
    for corr in (0.0095, 0.037, 0.072):
        case, e = _steady(corr)
        m = case["mesh"]
        mean, _, q = e.quantity_stats(QTY_DISP_MAGNITUDE, [0.05, 0.95])
        z = m.xyz[:, 2]
        mid = (z > 0.04) & (z < 0.26)          # one diameter away from the fixed ends
        R = 0.02
        # long clamped membrane tube at the mean E and h: u_r = (1 - nu^2) p R^2 / (E h)
        p = case["pressure"]
        ref = (1 - case["nu"] ** 2) * p * R ** 2 / (0.7e6 * 4.0e-3)
        assert mean[mid].mean() == pytest.approx(ref, rel=0.05)
        widths.append(float((q[mid, 1] - q[mid, 0]).mean()))
        e.close()
    assert widths[0] < widths[1] < widths[2], widths


def test_coarse_cylinder_two_realisations_against_oracle():
    case = synth.make_case("cylinder", level=0, corr=0.037, S=100, n_steps=401, seed=11)
    e = ens.Ensemble.from_case(case, precision="fp64")
    e.step(400)
    pick = [0, 99]
    u = e.displacement()[pick]
    ref = oracle.Model(case, samples=pick).run(400)[0]
    assert np.linalg.norm(u - ref) <= 1e-10 * np.linalg.norm(ref)
    e.close()
