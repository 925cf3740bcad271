"""Python binding of the ensemble solver's C ABI (argument marshalling only).

Every computation runs in libens.so (CUDA, sm_103a). PyTorch provides the device
memory (its caching allocator is handed to the library as the allocator hook) and the
stream the library launches on. Host arrays are numpy.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

FP64, FP32_FORCE, KAHAN32 = 0, 1, 2
FLAG_NO_AUTOTUNE, FLAG_UNSTAGED, FLAG_NO_GRAPH, FLAG_DEVICE_FIELDS = 1, 2, 4, 16
FLAG_ELEMENT_COEFFS = 32
QTY_DISPLACEMENT, QTY_DISP_MAGNITUDE, QTY_STRESS, QTY_PEAK_MAGNITUDE = 0, 1, 2, 3


def FLAG_FORCE_VARIANT(k: int) -> int:
    """Creation flag: use launch shape k (ens_info_t.kernel_variant) without autotuning."""
    return (k + 1) << 8
PRECISIONS = {"fp64": FP64, "fp32_force": FP32_FORCE, "kahan32": KAHAN32}
LAYOUT_SNC, LAYOUT_NCS = 0, 1


class EnsError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _torch():
    import torch
    return torch


class _TorchAllocator:
    """Adapter giving the library PyTorch's caching allocator on one device."""

    def __init__(self, device: int):
        torch = _torch()
        self.device = device
        self.sizes = {}

        def alloc(nbytes, stream, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=device,
                                                       stream=int(stream or 0))
                return int(p)
            except Exception:  # an exception may not cross into C
                return None

        def release(ptr, nbytes, stream, user):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._alloc = _lib.ALLOC_FN(alloc)
        self._release = _lib.RELEASE_FN(release)
        self.struct = _lib.ens_allocator(self._alloc, self._release, None)


def _check(L, ctx, rc):
    if rc != 0:
        msg = L.ens_last_error(ctx).decode() if ctx else ""
        if not msg:
            msg = L.ens_error_string(rc).decode()
        raise EnsError(rc, msg)


class Ensemble:
    """S realisations of the wall model advanced together on one GPU.

    xyz [N][3], tri [E][3], fixed [N][3] (uint8), E_node / h_node [N][S] (float64 host
    arrays, or float64 CUDA tensors on the context's device, e.g. from FieldSampler),
    material constants and dt as in ens_params; precision: "fp64", "fp32_force",
    "kahan32" or the ENS_* value. stream: a torch.cuda.Stream (default: current).
    """

    def __init__(self, xyz, tri, fixed, E_node, h_node, *, rho, nu, kshear, alpha, dt,
                 precision="fp64", stream=None, torch_allocator: bool = True, device: int = 0,
                 flags: int = 0, element_coeffs: bool = False):
        torch = _torch()
        self._L = _lib.load()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.fixed = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        on_device = isinstance(E_node, torch.Tensor) and E_node.is_cuda
        if on_device:
            for t in (E_node, h_node):
                assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                assert t.is_contiguous() and t.device.index == device and t.shape == E_node.shape
            flags |= FLAG_DEVICE_FIELDS
            fields = (ctypes.c_void_p(E_node.data_ptr()), ctypes.c_void_p(h_node.data_ptr()))
        else:
            E_node = np.ascontiguousarray(E_node, dtype=np.float64)
            h_node = np.ascontiguousarray(h_node, dtype=np.float64)
            fields = (_ptr(E_node), _ptr(h_node))
        if element_coeffs:  # E_node, h_node are (E h) and rho * hbar per element [E][S]
            flags |= FLAG_ELEMENT_COEFFS
        self.N, self.E = self.xyz.shape[0], self.tri.shape[0]
        self.S = int(E_node.shape[1])
        self.precision = PRECISIONS.get(precision, precision)
        self.device = device
        with torch.cuda.device(device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._allocator = _TorchAllocator(device) if torch_allocator else None
        mesh = _lib.ens_mesh(self.N, self.E, self.xyz.ctypes.data, self.tri.ctypes.data,
                             None if self.fixed is None else self.fixed.ctypes.data)
        params = _lib.ens_params(rho, nu, kshear, alpha, dt, int(self.precision), int(flags))
        out = ctypes.c_void_p()
        alloc_p = ctypes.byref(self._allocator.struct) if self._allocator else None
        with torch.cuda.device(device):
            if on_device:
                torch.cuda.current_stream(device).synchronize()  # the fields are written
            rc = self._L.ens_create(ctypes.byref(mesh), self.S, fields[0], fields[1],
                                    ctypes.byref(params), ctypes.c_void_p(self.stream.cuda_stream),
                                    alloc_p, ctypes.byref(out))
        if rc != 0:
            msg = self._L.ens_last_error(None).decode() or self._L.ens_error_string(rc).decode()
            raise EnsError(rc, msg)
        self._ctx = out

    @classmethod
    def from_case(cls, case, precision="fp64", **kw):
        """Build from a workload dict with keys mesh, E, h, rho, nu, kshear, alpha, dt,
        modes, amp (the traction table is set too)."""
        m = case["mesh"]
        ens = cls(m.xyz, m.tri, m.fixed, case["E"], case["h"], rho=case["rho"], nu=case["nu"],
                  kshear=case["kshear"], alpha=case["alpha"], dt=case["dt"], precision=precision,
                  **kw)
        ens.set_traction(case["modes"], case["amp"])
        return ens

    # -- life cycle ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            self._L.ens_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _call(self, name, *args):
        _check(self._L, self._ctx, getattr(self._L, name)(self._ctx, *args))

    # -- ABI calls ------------------------------------------------------------------
    def set_traction(self, modes, amp):
        modes = np.ascontiguousarray(modes, dtype=np.float64)
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        if modes.ndim != 3 or modes.shape[1:] != (self.N, 3) or amp.ndim != 2 or amp.shape[1] != modes.shape[0]:
            raise ValueError("modes must be [J][N][3] and amp [n_steps][J]")
        self._call("ens_set_traction", modes.shape[0], _ptr(modes), amp.shape[0], _ptr(amp))

    def set_amplitudes(self, first_row: int, amp):
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        self._call("ens_set_amplitudes", int(first_row), amp.shape[0], _ptr(amp))

    def step(self, n: int = 1):
        self._call("ens_step", int(n))

    def reset(self):
        self._call("ens_reset")

    def displacement(self, layout: str = "snc") -> np.ndarray:
        lay = LAYOUT_SNC if layout == "snc" else LAYOUT_NCS
        shape = (self.S, self.N, 3) if lay == LAYOUT_SNC else (self.N, 3, self.S)
        out = np.empty(shape, dtype=np.float64)
        self._call("ens_get_displacement", _ptr(out), lay)
        return out

    def displacement_device(self, out, layout: str = "snc"):
        """Write u_n into a float64 CUDA tensor (asynchronous on the context stream)."""
        lay = LAYOUT_SNC if layout == "snc" else LAYOUT_NCS
        assert out.is_cuda and out.dtype == _torch().float64 and out.numel() == self.S * self.N * 3
        self._call("ens_get_displacement_device", ctypes.c_void_p(out.data_ptr()), lay)
        return out

    def stats(self):
        mean = np.empty((self.N, 3))
        var = np.empty((self.N, 3))
        self._call("ens_stats", _ptr(mean), _ptr(var))
        return mean, var

    def stats_device(self, mean, var):
        self._call("ens_stats_device", ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(var.data_ptr()))
        return mean, var

    def internal_force(self, u_ncs) -> np.ndarray:
        u = np.ascontiguousarray(u_ncs, dtype=np.float64)
        assert u.shape == (self.N, 3, self.S)
        f = np.empty_like(u)
        self._call("ens_internal_force", _ptr(u), _ptr(f))
        return f

    def coefficients(self):
        eh = np.empty((self.E, self.S))
        minv = np.empty((self.N, self.S))
        self._call("ens_get_coefficients", _ptr(eh), _ptr(minv))
        return eh, minv

    def element_matrices(self) -> np.ndarray:
        k = np.empty((self.E, 9, 9))
        self._call("ens_get_element_matrices", _ptr(k))
        return k

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        self._call("ens_state_size", ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        self._call("ens_get_state", buf, n.value)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._call("ens_set_state", buf, len(blob))

    # -- output statistics (Section 3) -------------------------------------------
    def set_centerline(self, pts):
        """Centreline polyline [n][3] of the stress frame (Section 2.2.3)."""
        pts = np.ascontiguousarray(pts, dtype=np.float64)
        assert pts.ndim == 2 and pts.shape[1] == 3
        self._call("ens_set_centerline", pts.shape[0], _ptr(pts))

    def quantity_rows(self, qty: int) -> int:
        return {QTY_DISPLACEMENT: 3 * self.N, QTY_DISP_MAGNITUDE: self.N, QTY_STRESS: 6 * self.E,
                QTY_PEAK_MAGNITUDE: self.N}[qty]

    def quantity_device(self, qty: int, out=None):
        """Rows of a quantity at the current step as a CUDA float64 tensor [rows][S]."""
        torch = _torch()
        rows = self.quantity_rows(qty)
        if out is None:
            out = torch.empty((rows, self.S), dtype=torch.float64, device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == rows * self.S
        self._call("ens_quantity_device", int(qty), ctypes.c_void_p(out.data_ptr()))
        return out

    def quantity_stats(self, qty: int, q=()):
        """(mean [rows], variance [rows], quantiles [rows][len(q)] or None) of a quantity."""
        rows = self.quantity_rows(qty)
        qa = np.ascontiguousarray(q, dtype=np.float64)
        mean, var = np.empty(rows), np.empty(rows)
        quant = np.empty((rows, len(qa))) if len(qa) else None
        self._call("ens_quantity_stats", int(qty), len(qa), _ptr(qa) if len(qa) else None, _ptr(mean), _ptr(var),
                   _ptr(quant) if quant is not None else None)
        return mean, var, quant

    def set_geometry_update(self, k: int):
        """Re-assemble every realisation's stiffness on its deformed surface every k steps
        (Section 2.3); k = 0 returns to the linear method."""
        self._call("ens_set_geometry_update", int(k))

    def set_peak(self, stride: int = 1):
        """Track the running peak of |u| per node and realisation on every step index that
        is a multiple of stride (0: off); read it with QTY_PEAK_MAGNITUDE."""
        self._call("ens_set_peak", int(stride))

    def set_probes(self, nodes=(), elems=(), stride: int = 0, capacity: int = 0):
        """Record displacement at probe nodes and stress at probe elements every stride steps."""
        n = np.ascontiguousarray(nodes, dtype=np.int32)
        e = np.ascontiguousarray(elems, dtype=np.int32)
        self._probe_sizes = (n.size, e.size)
        self._call("ens_set_probes", n.size, _ptr(n) if n.size else None, e.size, _ptr(e) if e.size else None,
                   int(stride), int(capacity))

    def probes(self):
        """(steps [n_rec], u [n_rec][n_nodes][3][S], sigma [n_rec][n_elems][6][S])."""
        nn, ne = getattr(self, "_probe_sizes", (0, 0))
        n_rec = ctypes.c_int64()
        self._call("ens_get_probes", None, None, None, ctypes.byref(n_rec))
        r = n_rec.value
        u = np.empty((r, nn, 3, self.S))
        sig = np.empty((r, ne, 6, self.S))
        steps = np.empty(r, dtype=np.int64)
        self._call("ens_get_probes", _ptr(u) if u.size else None, _ptr(sig) if sig.size else None,
                   _ptr(steps) if r else None, ctypes.byref(n_rec))
        return steps, u, sig

    def info(self) -> dict:
        i = _lib.ens_info_t()
        self._call("ens_info", ctypes.byref(i))
        out = {name: getattr(i, name) for name, _ in i._fields_}
        out["variant_us"] = list(out["variant_us"])
        return out


BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT, BATCH_SEQUENCE = 0, 1, 2, 3


class Batch:
    """Several Ensembles (uneven meshes, widths and time steps; one precision form)
    advanced together by one batched launch per step (graph-captured) or one persistent
    launch (ens_batch_* in the C ABI). The members must outlive the batch."""

    def __init__(self, members, mode: int = BATCH_AUTO):
        self._L = _lib.load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._ctx.value for m in self.members])
        out = ctypes.c_void_p()
        rc = self._L.ens_batch_create(arr, len(self.members), int(mode), ctypes.byref(out))
        if rc != 0:
            msg = self._L.ens_last_error(self.members[0]._ctx).decode() or self._L.ens_error_string(rc).decode()
            raise EnsError(rc, msg)
        self._b = out

    def _check(self, rc):
        if rc != 0:
            raise EnsError(rc, self._L.ens_batch_last_error(self._b).decode())

    def step(self, n: int = 1):
        self._check(self._L.ens_batch_step(self._b, int(n)))

    def info(self) -> dict:
        i = _lib.ens_batch_info_t()
        self._check(self._L.ens_batch_info(self._b, ctypes.byref(i)))
        out = {name: getattr(i, name) for name, _ in i._fields_}
        out["mode_us"] = list(out["mode_us"])
        return out

    def close(self):
        if getattr(self, "_b", None):
            self._L.ens_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def merge_stats(parts):
    """Statistics of the union of disjoint sample shards: parts = [(count, mean, var), ...]
    with mean/var arrays of one shape (var: divisor count - 1). Runs ens_merge_stats."""
    L = _lib.load()
    k = len(parts)
    shape = np.shape(parts[0][1])
    means = [np.ascontiguousarray(p[1], dtype=np.float64).ravel() for p in parts]
    vars_ = [np.ascontiguousarray(p[2], dtype=np.float64).ravel() for p in parts]
    n = means[0].size
    counts = (ctypes.c_int64 * k)(*[int(p[0]) for p in parts])
    mp = (ctypes.c_void_p * k)(*[m.ctypes.data for m in means])
    vp = (ctypes.c_void_p * k)(*[v.ctypes.data for v in vars_])
    mo = np.empty(n)
    vo = np.empty(n)
    rc = L.ens_merge_stats(k, counts, mp, vp, n, _ptr(mo), _ptr(vo))
    if rc != 0:
        raise EnsError(rc, L.ens_error_string(rc).decode())
    return mo.reshape(shape), vo.reshape(shape)


def sharded_stats(count, mean, var, group=None):
    """Merge one rank's shard statistics with every other rank's: an all-gather of
    (count, mean, var) over torch.distributed, then ens_merge_stats on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    m = torch.as_tensor(np.ascontiguousarray(mean, dtype=np.float64), device=dev)
    v = torch.as_tensor(np.ascontiguousarray(var, dtype=np.float64), device=dev)
    c = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    ms = [torch.empty_like(m) for _ in range(world)]
    vs = [torch.empty_like(v) for _ in range(world)]
    cs = [torch.empty_like(c) for _ in range(world)]
    dist.all_gather(ms, m, group=group)
    dist.all_gather(vs, v, group=group)
    dist.all_gather(cs, c, group=group)
    parts = [(int(cc.item()), mm.cpu().numpy(), vv.cpu().numpy()) for cc, mm, vv in zip(cs, ms, vs)]
    return merge_stats(parts)


def row_stats_device(rows, q=(), stream=None):
    """Mean, sample variance and type-7 quantiles of every row of a CUDA float64 tensor
    [n_rows][S] (ens_row_stats_device); returns CUDA tensors (mean, var, quant or None)."""
    torch = _torch()
    L = _lib.load()
    assert rows.is_cuda and rows.dtype == torch.float64 and rows.is_contiguous() and rows.dim() == 2
    n, S = rows.shape
    qa = np.ascontiguousarray(q, dtype=np.float64)
    mean = torch.empty(n, dtype=torch.float64, device=rows.device)
    var = torch.empty_like(mean)
    quant = torch.empty((n, len(qa)), dtype=torch.float64, device=rows.device) if len(qa) else None
    st = stream if stream is not None else torch.cuda.current_stream(rows.device)
    rc = L.ens_row_stats_device(n, S, ctypes.c_void_p(rows.data_ptr()), len(qa), _ptr(qa) if len(qa) else None,
                                ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(var.data_ptr()),
                                ctypes.c_void_p(quant.data_ptr()) if quant is not None else None,
                                ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise EnsError(rc, L.ens_error_string(rc).decode())
    return mean, var, quant
