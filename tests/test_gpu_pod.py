"""Device POD (sur_pod) against the FP64 oracle (oracle/pod.py) on the same binary32
snapshots.

Tolerances: the device forms the Gram matrix from binary32 products summed 32 at a time
(relative error of a few 1e-7 of the entries), so eigenvalues agree within 1e-6 of the
largest; the rank-r reconstruction coef phi^T, which does not depend on signs or on the
basis of clustered modes, within 1e-5 (relative Frobenius norm); single modes with
well-separated eigenvalues within 1e-4 of their largest entry; the stored binary32 modes
are orthonormal within 1e-5."""
import numpy as np
import pytest

from oracle import pod as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_09059_gb300 import surrogate as sur  # noqa: E402


def _snapshots(n, D, s, noise, seed):
    rng = np.random.default_rng(seed)
    q = len(s)
    A = rng.standard_normal((n, q))
    A -= A.mean(axis=0)
    U, _ = np.linalg.qr(A)
    W, _ = np.linalg.qr(rng.standard_normal((D, q)))
    X = 1e-3 * rng.standard_normal(D)[None, :] + (U * np.asarray(s)[None, :]) @ W.T
    X += noise * rng.standard_normal((n, D))
    return X.astype(np.float32)


def _check(X, r, separated):
    Xd = torch.from_numpy(X).cuda()
    mean, phi, coef, lam, frac, iters = sur.pod_device(Xd, r)
    mean, phi, coef = mean.cpu().numpy(), phi.cpu().numpy(), coef.cpu().numpy()
    mo, po, co, lo, fo = op.pod(X.astype(np.float64), r)
    assert np.abs(mean - mo).max() <= 1e-6 * np.abs(mo).max()
    assert np.abs(lam - lo).max() <= 1e-6 * lo[0]
    assert frac == pytest.approx(fo, abs=1e-6)
    rec, rec_o = coef.astype(np.float64) @ phi.T.astype(np.float64), co @ po.T
    assert np.linalg.norm(rec - rec_o) <= 1e-5 * np.linalg.norm(X - mo)
    for k in separated:
        assert np.abs(phi[:, k] - po[:, k]).max() <= 1e-4 * np.abs(po[:, k]).max(), k
        assert np.abs(coef[:, k] - co[:, k]).max() <= 1e-4 * np.abs(co[:, k]).max(), k
    keep = lam > 1e-10 * lam[0]
    G = phi[:, keep].T.astype(np.float64) @ phi[:, keep].astype(np.float64)
    assert np.abs(G - np.eye(G.shape[0])).max() <= 1e-5
    return iters


def test_pod_matches_oracle_on_structured_snapshots():
    s = [40.0, 20.0, 11.0, 6.0, 3.5, 2.0, 1.1, 0.6, 0.3, 0.2]
    X = _snapshots(300, 5000, s, 1e-3, seed=1)
    iters = _check(X, 8, separated=range(8))
    assert 1 <= iters < 1000


def test_pod_of_rank_deficient_snapshots():
    """Rank-3 snapshots with r = 6: the block orthonormalisation meets dependent columns
    (Gram-Schmidt with refill), the surplus eigenvalues sit at the Gram matrix's rounding
    level and their modes stay finite."""
    X = _snapshots(64, 2000, [5.0, 2.0, 0.5], 0.0, seed=2)
    Xd = torch.from_numpy(X).cuda()
    mean, phi, coef, lam, frac, _ = sur.pod_device(Xd, 6)
    assert np.all(lam[3:] <= 1e-6 * lam[0])       # the Gram matrix's rounding, at most
    assert frac == pytest.approx(1.0, abs=1e-6)
    assert np.all(np.isfinite(phi.cpu().numpy())) and np.all(np.isfinite(coef.cpu().numpy()))
    _check(X, 3, separated=range(3))


def test_pod_rejects_bad_sizes():
    X = torch.zeros((4, 10), dtype=torch.float32, device="cuda")
    for r in (0, 4, 49):
        with pytest.raises(sur.EnsError):
            sur.pod_device(X, r)
