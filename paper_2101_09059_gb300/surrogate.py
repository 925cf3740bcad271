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


def pod(snapshots, r):
    """POD of snapshot rows: (mean [D], modes phi [D][r] orthonormal, coefficients [n][r],
    captured fraction of the fluctuation energy). Host linear algebra (set-up, not the
    time loop): eigenpairs of the snapshot Gram matrix."""
    X = np.asarray(snapshots, dtype=np.float32)
    mean = X.mean(axis=0, dtype=np.float64)
    Xc = X - mean.astype(np.float32)[None, :]
    G = (Xc @ Xc.T).astype(np.float64)
    w, V = np.linalg.eigh(G)
    order = np.argsort(-w)
    w, V = w[order], V[:, order]
    sig = np.sqrt(np.maximum(w[:r], 1e-300))
    phi = (Xc.T.astype(np.float64) @ V[:, :r]) / sig[None, :]
    coef = V[:, :r] * sig[None, :]
    frac = float(w[:r].sum() / max(w.sum(), 1e-300))
    return mean, np.ascontiguousarray(phi), np.ascontiguousarray(coef), frac
