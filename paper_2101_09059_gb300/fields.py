"""Python binding of the device Matérn field sampler (include/gmrf.h): argument
marshalling only. z and the output are float64 CUDA tensors [n_nodes][S] from PyTorch;
the assembly of K = kappa^2 C~ + G runs in the library's host code, the solves on the GPU."""
from __future__ import annotations

import ctypes
import numpy as np

from . import _lib
from .ensemble import EnsError


class FieldSampler:
    """x = K^-1 C~^(1/2) z on one surface mesh (Section 2.1, nu = 1), all samples at once."""

    def __init__(self, xyz, tri, corr_length: float, stream=None):
        import torch
        self._L = _lib.load()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.n_nodes = self.xyz.shape[0]
        self.corr_length = float(corr_length)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        out = ctypes.c_void_p()
        rc = self._L.gmrf_create(self.n_nodes, self.tri.shape[0], ctypes.c_void_p(self.xyz.ctypes.data),
                                 ctypes.c_void_p(self.tri.ctypes.data), self.corr_length,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out))
        if rc != 0:
            raise EnsError(rc, self._L.gmrf_last_error(None).decode())
        self._g = out
        self.kappa = self.info()["kappa"]

    def sample(self, z, sigma: float = 0.0, mean: float = 0.0, lognormal: bool = False,
               rtol: float = 1e-10, max_iter: int = 20000, out=None):
        """Fields from standard normals z (CUDA float64 [n_nodes][S]); returns out.
        sigma > 0: marginal standard deviation of the Gaussian field; sigma <= 0: x itself."""
        import torch
        assert z.is_cuda and z.dtype == torch.float64 and z.is_contiguous() and z.shape[0] == self.n_nodes
        S = z.shape[1]
        if out is None:
            out = torch.empty_like(z)
        rc = self._L.gmrf_sample(self._g, S, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 float(sigma), float(mean), 1 if lognormal else 0, float(rtol), int(max_iter))
        if rc != 0:
            raise EnsError(rc, self._L.gmrf_last_error(self._g).decode())
        return out

    def info(self) -> dict:
        i = _lib.gmrf_info_t()
        rc = self._L.gmrf_info(self._g, ctypes.byref(i))
        if rc != 0:
            raise EnsError(rc, self._L.gmrf_last_error(self._g).decode())
        return {k: getattr(i, k) for k, _ in i._fields_}

    def close(self):
        if getattr(self, "_g", None):
            self._L.gmrf_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
