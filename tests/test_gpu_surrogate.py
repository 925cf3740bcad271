"""GPU surrogate network (BF16 tensor-core products, FP32 state) against the FP64
oracle network (oracle/mlp.py).

Tolerances: the products round their inputs to BF16 (8 significant bits, relative
error 2^-9 per input), so outputs and gradients agree with the FP64 oracle to about
1e-2 relative; tests use 3e-2 (relative L2 per tensor)."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2101_09059_gb300 as ens  # noqa: E402
from paper_2101_09059_gb300 import surrogate as sur  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ens.load()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


def _data(B, n_in=64, n_out=32, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, n_in))
    t = np.tanh(x[:, :n_out] * 0.7) + 0.1 * x[:, n_out:2 * n_out] ** 2 if n_in >= 2 * n_out else rng.standard_normal((B, n_out))
    return x, t


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("B", [1, 37, 256, 1000])
def test_forward_matches_oracle(B):
    net = sur.Surrogate(64, 256, 32, max_batch=1024, seed=3)
    P = net.params()
    x, _ = _data(B)
    y = net.forward(_dev(x)).cpu().numpy()
    y_ref, _ = mlp.forward(P, x.astype(np.float32).astype(np.float64))
    assert rel(y, y_ref) < 3e-2
    net.close()


def test_gradients_match_oracle():
    net = sur.Surrogate(64, 256, 32, max_batch=512, seed=5)
    P = net.params()
    x, t = _data(300, seed=2)
    loss, g = net.loss_grad(_dev(x), _dev(t))
    L_ref, g_ref = mlp.gradients(P, x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
    assert loss == pytest.approx(L_ref, rel=3e-2)
    for k, (a, b) in enumerate(zip(g, g_ref)):
        assert rel(a, b) < 3e-2, k
    net.close()


def test_adam_first_step():
    net = sur.Surrogate(64, 256, 32, max_batch=512, seed=7)
    P0 = net.params()
    x, t = _data(256, seed=4)
    _, g = net.loss_grad(_dev(x), _dev(t))
    net.adam_step(_dev(x), _dev(t), 1e-3)
    P1 = net.params()
    for a, b, gg in zip(P1, P0, g):
        d = a - b
        # the first bias-corrected Adam step is exactly -lr * g / (|g| + eps)
        expect = -1e-3 * gg / (np.abs(gg) + 1e-8)
        assert np.allclose(d, expect, rtol=2e-3, atol=2e-9)
    net.close()


def test_adam_steps_match_oracle_adam_on_device_gradients():
    """Five Adam steps on distinct mini-batches. Before each step the device's gradient of
    the current parameters is read back (sur_loss_grad runs the same kernels on the same
    data as sur_adam_step, so it is the gradient the step uses); the FP64 oracle's Adam is
    fed those gradients from the same initial FP32 parameters. After every step each
    parameter tensor must match: the moments are carried, the bias corrections use this
    step's t, and beta1 / beta2 are not swapped. Tolerance: 1e-4 of the accumulated update
    (FP32 moments, square root and division) plus a few FP32 ulps of the parameter per step
    (the device stores the parameters in FP32)."""
    net = sur.Surrogate(64, 256, 32, max_batch=512, seed=13)
    P0 = net.params()
    P_orc = [p.copy() for p in P0]
    opt = mlp.Adam(P_orc, lr=2e-3)
    for t in range(1, 6):
        x, tg = _data(192, seed=20 + t)
        X, T = _dev(x), _dev(tg)
        _, g = net.loss_grad(X, T)
        net.adam_step(X, T, 2e-3)
        opt.step(P_orc, [np.asarray(gg, dtype=np.float64) for gg in g])
        P_dev = net.params()
        for k, (pd, po, p0) in enumerate(zip(P_dev, P_orc, P0)):
            tol = 1e-4 * np.abs(po - p0) + 2.0 * t * np.finfo(np.float32).eps * np.abs(po) + 1e-12
            assert np.all(np.abs(pd - po) <= tol), (t, k, float(np.abs(pd - po).max()))
    net.close()


def test_training_reduces_loss_like_the_oracle():
    x, t = _data(2048, seed=9)
    net = sur.Surrogate(64, 256, 32, max_batch=2048, seed=11)
    P = net.params()
    X, T = _dev(x), _dev(t)
    l0 = net.loss(X, T)
    hist = net.train(X, T, epochs=30, batch=256, lr=1e-3, seed=1)
    l1 = net.loss(X, T)
    assert hist.shape == (30,) and np.all(np.isfinite(hist))
    assert l1 < 0.2 * l0
    # the FP64 oracle, same initial weights and data, full-batch Adam for a few steps,
    # ends at a loss of the same order
    opt = mlp.Adam(P, lr=1e-3)
    xr, tr = x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)
    for _ in range(240):
        _, gr = mlp.gradients(P, xr, tr)
        opt.step(P, gr)
    l_ref = mlp.loss(P, xr, tr)
    assert l1 < 5 * l_ref + 1e-3
    net.close()


def test_matmul_and_reconstruct():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((300, 1111))
    B = rng.standard_normal((1111, 40))
    C = sur.matmul(_dev(A), _dev(B)).cpu().numpy()
    assert rel(C, A @ B) < 1e-2
    Ct = sur.matmul(_dev(A.T.copy()), _dev(B.T.copy()), transpose_a=True, transpose_b=True).cpu().numpy()
    assert rel(Ct, A @ B) < 1e-2
    coef = rng.standard_normal((7, 5))
    mean = rng.standard_normal(1234)
    phi = rng.standard_normal((1234, 5))
    u = sur.reconstruct(_dev(coef), _dev(mean), _dev(phi)).cpu().numpy()
    assert rel(u, mean[None, :] + coef @ phi.T) < 1e-6


def test_surrogate_pipeline_beats_plain_ensemble_on_time_to_statistics():
    """Train the surrogate on solver runs of a small aneurysm tube and show what it gains:
    ensemble mean and standard-deviation fields of held-out realisations, from the network,
    match the solver's to within a few percent at a small fraction of the solver's time."""
    import time
    import synth
    m = synth.aneurysm_mesh(40, 50)
    basis = synth.kl_basis(m, 8)
    n_train, n_val, S = 1024, 256, 256
    xi = synth.kl_coefficients(n_train + n_val, 8, seed=5)
    E_all, h_all = synth.kl_fields(basis, xi)
    dt = synth.cfl_dt(m, E_all)
    n_steps = int(round(0.03 / dt))
    params = dict(rho=synth.configs.RHO, nu=synth.configs.NU, kshear=synth.configs.KSHEAR,
                  alpha=synth.configs.ALPHA, dt=dt)
    modes = synth.pressure_shear_modes(m, with_shear=True)
    amp = synth.peak_amplitudes(n_steps, dt)

    def fields_for(rows):
        return np.ascontiguousarray(E_all[:, rows]), np.ascontiguousarray(h_all[:, rows])

    U = sur.solver_fields(m, fields_for, n_train + n_val, S, params, modes, amp, n_steps)
    mean, phi, coef, frac = sur.pod(U[:n_train], 8)
    assert frac > 0.99
    cs = coef.std(axis=0)
    net = sur.Surrogate(16, 64, 8, max_batch=1024, seed=1)
    X, T = _dev(xi[:n_train]), _dev(coef / cs)
    for lr, ep in ((3e-3, 150), (1e-3, 150), (3e-4, 100)):
        net.train(X, T, epochs=ep, batch=128, lr=lr, seed=ep)
    net.scale_outputs(cs)              # predictions in POD coefficient units
    # held-out realisations; the trained surrogate's basis lives on the device
    Xv, mean_d, phi_d = _dev(xi[n_train:]), _dev(mean), _dev(phi)
    for _ in range(2):                 # the second, warm pass is timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cpred = net.forward(Xv)
        mu_s, sd_s = sur.field_stats(cpred, mean_d, phi_d)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t0
    t0 = time.perf_counter()
    Uv = sur.solver_fields(m, lambda rows: fields_for([n_train + r for r in rows]), n_val, S, params, modes,
                           amp, n_steps)
    t_solver = time.perf_counter() - t0
    mu_ref, sd_ref = Uv.mean(axis=0), Uv.std(axis=0, ddof=1)
    e_mean = rel(mu_s.cpu().numpy(), mu_ref)
    e_std = rel(sd_s.cpu().numpy(), sd_ref)
    upred = sur.reconstruct(cpred, mean_d, phi_d).cpu().numpy()
    e_fluct = rel(upred - mu_ref[None, :], Uv - mu_ref[None, :])
    print(f"surrogate: mean {e_mean:.2e} std {e_std:.2e} fluctuation {e_fluct:.2e} "
          f"time {t_sur * 1e3:.2f} ms vs solver {t_solver * 1e3:.0f} ms")
    assert e_mean < 1e-2 and e_std < 0.15 and e_fluct < 0.35
    assert t_sur < 0.1 * t_solver
    net.close()


def test_untrusted_realisations_fall_back_to_the_solver():
    """The plain solver is the surrogate's fallback: inputs outside the trust radius (the
    0.99-quantile of the training inputs' norms) are flagged, and their fields in the
    pipeline's output are the solver's, bit for bit; trusted rows are the network's
    reconstruction. Four of the twelve test inputs are training-like draws scaled by 4
    (norm about 11 against a radius near 4.5 for 8 standard-normal coefficients)."""
    import synth
    m = synth.aneurysm_mesh(24, 30)
    basis = synth.kl_basis(m, 4)
    n_train, S = 256, 64
    xi = synth.kl_coefficients(n_train, 4, seed=9)
    E_all, h_all = synth.kl_fields(basis, xi)
    xt = synth.kl_coefficients(12, 4, seed=10)
    xt[8:] *= 4.0
    E_t, h_t = synth.kl_fields(basis, xt)
    dt = synth.cfl_dt(m, np.concatenate([E_all, E_t], axis=1))
    n_steps = int(round(0.01 / dt))
    params = dict(rho=synth.configs.RHO, nu=synth.configs.NU, kshear=synth.configs.KSHEAR,
                  alpha=synth.configs.ALPHA, dt=dt)
    modes = synth.pressure_shear_modes(m, with_shear=True)
    amp = synth.peak_amplitudes(n_steps, dt)
    U = sur.solver_fields(m, lambda r: (E_all[:, r].copy(), h_all[:, r].copy()), n_train, S, params, modes,
                          amp, n_steps)
    mean, phi, coef, _ = sur.pod(U, 4)
    cs = coef.std(axis=0)
    net = sur.Surrogate(8, 32, 4, max_batch=256, seed=2)
    X = _dev(xi)
    net.train(X, _dev(coef / cs), epochs=60, batch=64, lr=3e-3, seed=1)
    net.scale_outputs(cs)
    radius = net.fit_trust(X, 0.99)
    norms = np.sort(np.linalg.norm(xi.astype(np.float32).astype(np.float64), axis=1))
    assert radius == pytest.approx(norms[int(np.ceil(0.99 * n_train)) - 1], rel=1e-12)

    def solve(rows):
        return sur.solver_fields(m, lambda r: (E_t[:, rows[r]].copy(), h_t[:, rows[r]].copy()), len(rows), S,
                                 params, modes, amp, n_steps)

    Xt, mean_d, phi_d = _dev(xt), _dev(mean), _dev(phi)
    u, trusted = sur.predict_with_fallback(net, Xt, mean_d, phi_d, solve)
    trusted = trusted.cpu().numpy()
    expect = np.linalg.norm(xt.astype(np.float32).astype(np.float64), axis=1) <= radius
    assert np.array_equal(trusted, expect) and not trusted[8:].any() and trusted[:8].sum() >= 6
    u = u.cpu().numpy()
    bad = np.flatnonzero(~trusted)
    assert np.array_equal(u[bad], solve(bad))
    plain = sur.reconstruct(net.forward(Xt), mean_d, phi_d).cpu().numpy()
    assert np.array_equal(u[trusted], plain[trusted])
    with pytest.raises(ens.EnsError):
        sur.Surrogate(8, 32, 4, max_batch=16, seed=3).trusted(Xt)     # no radius fitted yet
    net.close()


def _bf16(a):
    """Round float32 values to BF16 (nearest, ties to even) and back, in numpy."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 64, 32), (129, 65, 33), (300, 200, 1111), (256, 256, 16)])
def test_tensor_core_product_equals_bf16_inputs_with_fp32_accumulation(M, N, K):
    """The product of the BF16-rounded operands, accumulated in binary64. Products of BF16
    values are exact in FP32; the device's FP32 accumulation over K terms may differ from
    the exact sum by (K + 2) * 2^-22 of the sum of |terms| (a bound that also covers an
    accumulator that truncates instead of rounding)."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    C = sur.matmul(_dev(A), _dev(B)).cpu().numpy().astype(np.float64)
    Ab, Bb = _bf16(A), _bf16(B)
    ref = Ab @ Bb
    bound = (K + 2) * 2.0 ** -22 * (np.abs(Ab) @ np.abs(Bb)) + 1e-30
    assert np.all(np.abs(C - ref) <= bound)
