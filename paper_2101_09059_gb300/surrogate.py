"""Python binding of the surrogate network's C ABI (include/sur.h): argument
marshalling only. Device arrays are float32 CUDA tensors from PyTorch; the forward and
backward passes, the optimiser and the POD products run in libens.so."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .ensemble import EnsError


def _dp(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_f32(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()


class Surrogate:
    """GELU MLP n_in -> hidden -> hidden -> n_out, BF16 tensor-core products, FP32 state."""

    def __init__(self, n_in=64, hidden=256, n_out=32, max_batch=4096, seed=0, stream=None):
        import torch
        self._L = _lib.load()
        self.n_in, self.hidden, self.n_out, self.max_batch = n_in, hidden, n_out, max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        out = ctypes.c_void_p()
        rc = self._L.sur_create(n_in, hidden, n_out, max_batch, seed,
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out))
        if rc != 0:
            raise EnsError(rc, "sur_create failed")
        self._c = out
        self.n_params = int(self._L.sur_param_count(self._c))
        offs = (ctypes.c_int64 * 6)()
        self._chk(self._L.sur_param_offsets(self._c, offs))
        self.offsets = list(offs)
        self.shapes = [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,)]

    def _chk(self, rc):
        if rc != 0:
            raise EnsError(rc, self._L.sur_last_error(self._c).decode())

    # -- parameters -------------------------------------------------------------------
    def get_flat(self) -> np.ndarray:
        h = np.empty(self.n_params, dtype=np.float32)
        self._chk(self._L.sur_get_params(self._c, ctypes.c_void_p(h.ctypes.data)))
        return h

    def set_flat(self, flat):
        h = np.ascontiguousarray(flat, dtype=np.float32)
        assert h.size == self.n_params
        self._chk(self._L.sur_set_params(self._c, ctypes.c_void_p(h.ctypes.data)))

    def unflatten(self, flat):
        return [np.asarray(flat[o:o + int(np.prod(s))], dtype=np.float64).reshape(s)
                for o, s in zip(self.offsets, self.shapes)]

    def flatten(self, tensors):
        flat = np.zeros(self.n_params, dtype=np.float32)
        for o, t in zip(self.offsets, tensors):
            flat[o:o + t.size] = np.asarray(t, dtype=np.float32).ravel()
        return flat

    def params(self):
        return self.unflatten(self.get_flat())

    def set_params(self, tensors):
        self.set_flat(self.flatten(tensors))

    # -- compute ----------------------------------------------------------------------
    def forward(self, x, out=None):
        import torch
        _check_f32(x)
        if out is None:
            out = torch.empty((x.shape[0], self.n_out), dtype=torch.float32, device=x.device)
        self._chk(self._L.sur_forward(self._c, _dp(x), x.shape[0], _dp(out)))
        return out

    def loss_grad(self, x, t):
        _check_f32(x)
        _check_f32(t)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.n_params, dtype=np.float32)
        self._chk(self._L.sur_loss_grad(self._c, _dp(x), _dp(t), x.shape[0],
                                        ctypes.c_void_p(loss.ctypes.data), ctypes.c_void_p(g.ctypes.data)))
        return float(loss[0]), self.unflatten(g)

    def loss(self, x, t) -> float:
        out = np.zeros(1, dtype=np.float32)
        self._chk(self._L.sur_loss(self._c, _dp(x), _dp(t), x.shape[0], ctypes.c_void_p(out.ctypes.data)))
        return float(out[0])

    def adam_step(self, x, t, lr):
        self._chk(self._L.sur_adam_step(self._c, _dp(x), _dp(t), x.shape[0], ctypes.c_float(lr)))

    def scale_outputs(self, scale):
        """Multiply the network's outputs by `scale` [n_out] by rescaling the last layer
        (exact): used to undo the target standardisation after training."""
        P = self.params()
        sc = np.asarray(scale, dtype=np.float64)
        P[4] = P[4] * sc[:, None]
        P[5] = P[5] * sc
        self.set_params(P)

    def train(self, X, T, epochs, batch=256, lr=1e-3, seed=0):
        _check_f32(X)
        _check_f32(T)
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        self._chk(self._L.sur_train(self._c, _dp(X), _dp(T), X.shape[0], batch, epochs, ctypes.c_float(lr),
                                    seed, ctypes.c_void_p(hist.ctypes.data)))
        return hist[:epochs]

    def fit_trust(self, X, q=0.99) -> float:
        """Trust radius from the training inputs X (CUDA float32 [n][n_in]): the q-quantile
        of their norms (sur_fit_trust); returns it."""
        _check_f32(X)
        r = ctypes.c_double()
        self._chk(self._L.sur_fit_trust(self._c, _dp(X), X.shape[0], float(q), ctypes.byref(r)))
        return r.value

    def trusted(self, x):
        """Bool CUDA tensor [B]: inputs within the trust radius (sur_trust)."""
        import torch
        _check_f32(x)
        flags = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
        self._chk(self._L.sur_trust(self._c, _dp(x), x.shape[0], _dp(flags)))
        return flags.bool()

    def close(self):
        if getattr(self, "_c", None):
            self._L.sur_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def matmul(A, B, transpose_a=False, transpose_b=False, out=None, stream=None):
    """out = op(A) @ op(B) on the tensor cores (BF16 inputs, FP32 accumulation)."""
    import torch
    L = _lib.load()
    _check_f32(A)
    _check_f32(B)
    M, K = (A.shape[1], A.shape[0]) if transpose_a else (A.shape[0], A.shape[1])
    K2, N = (B.shape[1], B.shape[0]) if transpose_b else (B.shape[0], B.shape[1])
    assert K == K2
    sam, sak = (1, A.shape[1]) if transpose_a else (A.shape[1], 1)
    sbk, sbn = (1, B.shape[1]) if transpose_b else (B.shape[1], 1)
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sur_matmul(_dp(A), sam, sak, _dp(B), sbk, sbn, _dp(out), M, N, K, N, ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise EnsError(rc, "sur_matmul failed")
    return out


def reconstruct(coef, mean, phi, out=None, stream=None):
    """out [B][D] = mean [D] + coef [B][r] phi [D][r]^T (FP32)."""
    import torch
    L = _lib.load()
    B, r = coef.shape
    D = mean.shape[0]
    if out is None:
        out = torch.empty((B, D), dtype=torch.float32, device=coef.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sur_reconstruct(_dp(coef), _dp(mean), _dp(phi), B, D, r, _dp(out), ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise EnsError(rc, "sur_reconstruct failed")
    return out


def field_stats(coef, mean, phi, stream=None):
    """(mean [D], std [D]) of u = mean + phi c over the coefficient rows coef [M][r]."""
    import torch
    L = _lib.load()
    M, r = coef.shape
    D = mean.shape[0]
    work = torch.empty(r + r * r, dtype=torch.float32, device=coef.device)
    m_out = torch.empty(D, dtype=torch.float32, device=coef.device)
    s_out = torch.empty(D, dtype=torch.float32, device=coef.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sur_field_stats(_dp(coef), M, r, _dp(mean), _dp(phi), D, _dp(work), _dp(m_out), _dp(s_out),
                           ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise EnsError(rc, "sur_field_stats failed")
    return m_out, s_out


# ---- pipeline: solver data -> POD -> training -> prediction ---------------------------

def solver_fields(mesh, fields_for, n_runs, S, params, modes, amp, n_steps, precision="kahan32",
                  stream=None, device=0):
    """Final displacements [n_runs][3N] (float32) of n_runs realisations, S per launch;
    fields_for(rows) returns the nodal (E, h) [N][len(rows)] of those realisations."""
    from .ensemble import Ensemble
    N = mesh.n_nodes
    out = np.empty((n_runs, 3 * N), dtype=np.float32)
    for r0 in range(0, n_runs, S):
        rows = list(range(r0, min(n_runs, r0 + S)))
        E, h = fields_for(rows)
        with Ensemble(mesh.xyz, mesh.tri, mesh.fixed, E, h, precision=precision, stream=stream,
                      device=device, **params) as e:
            e.set_traction(modes, amp)
            e.step(n_steps)
            out[r0:r0 + len(rows)] = e.displacement("snc").reshape(len(rows), -1)
    return out


def pod(snapshots, r, stream=None):
    """POD of snapshot rows on the device (sur_pod): (mean [D], modes phi [D][r]
    orthonormal, coefficients [n][r], captured fraction of the fluctuation energy) as
    numpy arrays. snapshots: numpy [n][D] or a CUDA float32 tensor."""
    import torch
    L = _lib.load()
    X = snapshots if isinstance(snapshots, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(snapshots, dtype=np.float32)).cuda()
    _check_f32(X)
    n, D = X.shape
    mean = torch.empty(D, dtype=torch.float32, device=X.device)
    phi = torch.empty((D, r), dtype=torch.float32, device=X.device)
    coef = torch.empty((n, r), dtype=torch.float32, device=X.device)
    frac = ctypes.c_double()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sur_pod(_dp(X), n, D, int(r), _dp(mean), _dp(phi), _dp(coef), None, ctypes.byref(frac), None,
                   ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise EnsError(rc, "sur_pod failed")
    return mean.cpu().numpy(), phi.cpu().numpy(), coef.cpu().numpy(), frac.value


def pod_device(X, r, stream=None):
    """sur_pod on a CUDA float32 tensor X [n][D]: (mean, phi, coef) CUDA tensors, the
    eigenvalues [r] and captured fraction (host), and the iterations taken."""
    import torch
    L = _lib.load()
    _check_f32(X)
    n, D = X.shape
    mean = torch.empty(D, dtype=torch.float32, device=X.device)
    phi = torch.empty((D, r), dtype=torch.float32, device=X.device)
    coef = torch.empty((n, r), dtype=torch.float32, device=X.device)
    lam = np.zeros(r)
    frac, iters = ctypes.c_double(), ctypes.c_int32()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.sur_pod(_dp(X), n, D, int(r), _dp(mean), _dp(phi), _dp(coef), ctypes.c_void_p(lam.ctypes.data),
                   ctypes.byref(frac), ctypes.byref(iters), ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise EnsError(rc, "sur_pod failed")
    return mean, phi, coef, lam, frac.value, iters.value

def predict_with_fallback(net, xi, mean, phi, solve):
    """Fields of the realisations xi [B][n_in] (CUDA float32): the network's prediction
    u = mean + phi c (sur_forward, sur_reconstruct) where the input lies within the trust
    radius (sur_trust), and the solver's own fields where it does not: solve(rows) runs the
    plain solver on those rows' realisations and returns their fields [len(rows)][D] (for
    example solver_fields), which are copied in unchanged. Returns (u [B][D] CUDA float32,
    trusted [B] bool)."""
    import torch
    u = reconstruct(net.forward(xi), mean, phi)
    trusted = net.trusted(xi)
    bad = torch.nonzero(~trusted).flatten()
    if bad.numel():
        fields = np.ascontiguousarray(solve(bad.cpu().numpy()), dtype=np.float32)
        u[bad] = torch.from_numpy(fields).to(u.device)
    return u, trusted
