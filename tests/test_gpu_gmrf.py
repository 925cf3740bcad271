"""Device Matérn field sampler (include/gmrf.h) against the FP64 oracle (oracle/gmrf.py).

The device solves K x = C~^(1/2) z by conjugate gradients to ||K x - b|| <= rtol ||b||;
the oracle solves it directly. Since G is positive semi-definite, K = kappa^2 C~ + G has
smallest eigenvalue >= kappa^2 min C~, so ||x - x*|| <= rtol ||b|| / (kappa^2 min C~):
that bound (times 2 for rounding in the residual recursion) is the tolerance."""
import numpy as np
import pytest

import oracle.gmrf as og
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_09059_gb300 as pkg  # noqa: E402

RHO = 0.02


def normals(n, S, seed):
    rng = np.random.Generator(np.random.Philox(key=seed))
    return rng.standard_normal((n, S))


def bound(m, z, rtol):
    kappa = og.kappa_of(RHO)
    Cl = og.lumped_mass(m.xyz, m.tri)
    b = np.sqrt(Cl)[:, None] * z
    return 2.0 * rtol * np.linalg.norm(b, axis=0) / (kappa ** 2 * Cl.min())


@pytest.mark.parametrize("S", [1, 7, 64])
def test_sampler_matches_direct_solve(S):
    m = synth.aneurysm_mesh(nc=40, na=30)
    z = normals(m.n_nodes, S, 5 + S)
    fs = pkg.FieldSampler(m.xyz, m.tri, RHO)
    rtol = 1e-10
    x = fs.sample(torch.from_numpy(z).cuda(), rtol=rtol).cpu().numpy()
    info = fs.info()
    assert info["max_relres"] <= rtol and info["iterations"] > 0
    ref = og.sample(m.xyz, m.tri, og.kappa_of(RHO), z)
    err = np.linalg.norm(x - ref, axis=0)
    assert np.all(err <= bound(m, z, rtol)), (err, bound(m, z, rtol))
    fs.close()


def test_lognormal_transform_and_determinism():
    m = synth.tube_mesh(nc=32, na=24, radius=0.01, length=0.06)
    S, sigma, mean = 9, 0.1, 0.7e6
    z = normals(m.n_nodes, S, 77)
    z[:, 4] = 0.0   # a zero draw: the field is exactly the mean
    fs = pkg.FieldSampler(m.xyz, m.tri, RHO)
    zt = torch.from_numpy(z).cuda()
    kappa = og.kappa_of(RHO)
    # the library derives kappa from the correlation length as the pinned oracle does
    assert fs.kappa == pytest.approx(kappa, rel=1e-15)
    scale = og.marginal_scale(kappa, sigma)
    a = fs.sample(zt, sigma=sigma, mean=mean, lognormal=True).cpu().numpy()
    b = fs.sample(zt, sigma=sigma, mean=mean, lognormal=True).cpu().numpy()
    assert np.array_equal(a, b)
    assert np.all(a[:, 4] == mean)
    x = og.sample(m.xyz, m.tri, kappa, z) * og.marginal_scale(kappa, sigma)
    ref = mean * np.exp(x)
    # |d exp(v)| <= exp(v) |dv| with |dv| <= scale * (solve bound), plus rounding of exp
    dv = scale * bound(m, z, 1e-10)
    assert np.all(np.abs(a - ref) <= ref * (dv[None, :] + 4e-16) * 1.01 + 1e-300)
    lin = fs.sample(zt, sigma=sigma, mean=1.0, lognormal=False).cpu().numpy()
    assert np.abs(lin - (1.0 + x)).max() <= dv.max() * 1.01 + 1e-15
    fs.close()


def test_iteration_limit_reports_not_converged():
    m = synth.aneurysm_mesh(nc=40, na=30)
    z = normals(m.n_nodes, 3, 9)
    fs = pkg.FieldSampler(m.xyz, m.tri, RHO)
    with pytest.raises(pkg.EnsError) as e:
        fs.sample(torch.from_numpy(z).cuda(), rtol=1e-12, max_iter=5)
    assert e.value.code == -9
    assert fs.info()["iterations"] == 5
    fs.close()


def test_device_fields_feed_the_ensemble_bitwise():
    """E and h drawn on the device and passed to ens_create as device arrays give the same
    trajectory, bit for bit, as the same values passed from the host."""
    case = synth.make_case("tube_small", S=6, n_steps=60, seed=0)
    m = case["mesh"]
    fs = pkg.FieldSampler(m.xyz, m.tri, RHO)
    zE = torch.from_numpy(normals(m.n_nodes, 6, 1)).cuda()
    zh = torch.from_numpy(normals(m.n_nodes, 6, 2)).cuda()
    E = fs.sample(zE, sigma=0.1, mean=0.7e6, lognormal=True)
    h = fs.sample(zh, sigma=0.1, mean=1e-3, lognormal=True)
    kw = dict(rho=case["rho"], nu=case["nu"], kshear=case["kshear"], alpha=case["alpha"], dt=case["dt"],
              precision="fp64")
    dev = pkg.Ensemble(m.xyz, m.tri, m.fixed, E, h, **kw)
    host = pkg.Ensemble(m.xyz, m.tri, m.fixed, E.cpu().numpy(), h.cpu().numpy(), **kw)
    for e in (dev, host):
        e.set_traction(case["modes"], case["amp"])
        e.step(50)
    assert np.array_equal(dev.displacement(), host.displacement())
    bad = E.clone()
    bad[3, 2] = -1.0
    with pytest.raises(pkg.EnsError):
        pkg.Ensemble(m.xyz, m.tri, m.fixed, bad, h, **kw)
    dev.close()
    host.close()
    fs.close()


def test_full_size_aneurysm_sampled():
    """200k-node aneurysm, S = 64 as the workload draws it; two samples against the oracle."""
    m = synth.aneurysm_mesh()
    S = 64
    z = normals(m.n_nodes, S, 123)
    fs = pkg.FieldSampler(m.xyz, m.tri, RHO)
    rtol = 1e-10
    x = fs.sample(torch.from_numpy(z).cuda(), rtol=rtol).cpu().numpy()
    assert fs.info()["max_relres"] <= rtol
    pick = [0, 63]
    ref = og.sample(m.xyz, m.tri, og.kappa_of(RHO), z[:, pick])
    err = np.linalg.norm(x[:, pick] - ref, axis=0)
    assert np.all(err <= bound(m, z[:, pick], rtol))
    fs.close()


def test_rows_longer_than_sixteen_take_the_csr_product():
    """A flat fan around one hub node of degree 24, so the hub's row of K holds 25 entries
    and the product runs over the CSR rows instead of the padded ones: the same bound
    against the oracle's direct solve."""
    n_ring = 24
    ang = 2.0 * np.pi * np.arange(n_ring) / n_ring
    ring1 = np.stack([0.01 * np.cos(ang), 0.01 * np.sin(ang), np.zeros(n_ring)], 1)
    a2 = ang + np.pi / n_ring
    ring2 = np.stack([0.02 * np.cos(a2), 0.02 * np.sin(a2), np.zeros(n_ring)], 1)
    xyz = np.vstack([[[0.0, 0.0, 0.0]], ring1, ring2])
    tri = []
    for k in range(n_ring):
        k1 = (k + 1) % n_ring
        tri.append([0, 1 + k, 1 + k1])
        tri.append([1 + k, 1 + n_ring + k, 1 + k1])
        tri.append([1 + k1, 1 + n_ring + k, 1 + n_ring + k1])
    tri = np.asarray(tri, dtype=np.int32)

    class Mesh:
        pass
    m = Mesh()
    m.xyz, m.tri, m.n_nodes = xyz, tri, xyz.shape[0]
    S, rtol = 6, 1e-10
    z = normals(m.n_nodes, S, 31)
    fs = pkg.FieldSampler(xyz, tri, RHO)
    x = fs.sample(torch.from_numpy(z).cuda(), rtol=rtol).cpu().numpy()
    assert fs.info()["max_relres"] <= rtol
    ref = og.sample(xyz, tri, og.kappa_of(RHO), z)
    err = np.linalg.norm(x - ref, axis=0)
    assert np.all(err <= bound(m, z, rtol)), (err, bound(m, z, rtol))
    fs.close()
