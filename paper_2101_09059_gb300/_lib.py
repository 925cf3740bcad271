"""Build and load the CUDA library (libens.so) and declare its C ABI for ctypes.

The library is compiled in-tree for sm_103a only; nothing here computes anything.
A missing or unloadable library raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libens.so")
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ens.h", "sur.h", "gmrf.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + HEADERS


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ (in parallel) and link libens.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        log = os.path.join(BUILD, os.path.basename(src)[:-3] + ".ptxas.txt")
        with open(log, "w") as fh:
            fh.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    return LIB


def declared_functions():
    """Names of the functions declared in include/*.h (for the export check)."""
    names = []
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b((?:ens|sur|gmrf)_[a-z0-9_]+)\s*\(", txt):
            names.append(m.group(1))
    return sorted(set(names))


class ens_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_elems", ctypes.c_int32),
                ("xyz", ctypes.c_void_p), ("tri", ctypes.c_void_p), ("fixed", ctypes.c_void_p)]


class ens_params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("nu", ctypes.c_double), ("kshear", ctypes.c_double),
                ("alpha", ctypes.c_double), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class ens_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", ctypes.c_void_p)]


class ens_info_t(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_elems", ctypes.c_int32),
                ("n_samples", ctypes.c_int32), ("n_samples_padded", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("n_steps_table", ctypes.c_int64), ("step", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("dt", ctypes.c_double), ("omega_lower", ctypes.c_double),
                ("omega_upper", ctypes.c_double), ("bytes_per_step", ctypes.c_double),
                ("device_bytes", ctypes.c_double), ("kernel_variant", ctypes.c_int32),
                ("variant_us", ctypes.c_float * 16)]


class ens_batch_info_t(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_int32), ("mode", ctypes.c_int32), ("block", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("n_tiles", ctypes.c_int32),
                ("persistent_grid", ctypes.c_int32), ("mode_us", ctypes.c_float * 5),
                ("bytes_per_step", ctypes.c_double)]


class gmrf_info_t(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("nnz", ctypes.c_int64), ("iterations", ctypes.c_int32),
                ("max_relres", ctypes.c_double), ("bytes_per_iter", ctypes.c_double),
                ("last_S", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("bytes_per_refinement", ctypes.c_double), ("kappa", ctypes.c_double)]


_lib = None


def load(build_if_missing: bool = True):
    """Load libens.so (building it first if allowed); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        build()
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library not built: {LIB}")
    L = ctypes.CDLL(LIB)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "ens_create": ([ctypes.POINTER(ens_mesh), i32, dp, dp, ctypes.POINTER(ens_params), vp,
                        ctypes.POINTER(ens_allocator), ctypes.POINTER(vp)], ctypes.c_int),
        "ens_set_traction": ([vp, i32, dp, i64, dp], ctypes.c_int),
        "ens_set_amplitudes": ([vp, i64, i64, dp], ctypes.c_int),
        "ens_step": ([vp, i64], ctypes.c_int),
        "ens_reset": ([vp], ctypes.c_int),
        "ens_get_displacement": ([vp, dp, i32], ctypes.c_int),
        "ens_get_displacement_device": ([vp, dp, i32], ctypes.c_int),
        "ens_stats": ([vp, dp, dp], ctypes.c_int),
        "ens_stats_device": ([vp, dp, dp], ctypes.c_int),
        "ens_internal_force": ([vp, dp, dp], ctypes.c_int),
        "ens_internal_force_noalloc": ([vp, dp, dp], ctypes.c_int),
        "ens_get_coefficients": ([vp, dp, dp], ctypes.c_int),
        "ens_get_element_matrices": ([vp, dp], ctypes.c_int),
        "ens_state_size": ([vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "ens_get_state": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
        "ens_set_state": ([vp, vp, ctypes.c_size_t], ctypes.c_int),
        "ens_info": ([vp, ctypes.POINTER(ens_info_t)], ctypes.c_int),
        "ens_last_error": ([vp], ctypes.c_char_p),
        "ens_error_string": ([ctypes.c_int], ctypes.c_char_p),
        "ens_destroy": ([vp], None),
        "ens_merge_stats": ([i32, ctypes.POINTER(i64), ctypes.POINTER(dp), ctypes.POINTER(dp), i64, dp, dp],
                            ctypes.c_int),
        "ens_batch_create": ([ctypes.POINTER(vp), i32, i32, ctypes.POINTER(vp)], ctypes.c_int),
        "ens_batch_step": ([vp, i64], ctypes.c_int),
        "ens_batch_info": ([vp, ctypes.POINTER(ens_batch_info_t)], ctypes.c_int),
        "ens_batch_last_error": ([vp], ctypes.c_char_p),
        "ens_batch_destroy": ([vp], None),
        "sur_create": ([i32, i32, i32, i32, ctypes.c_uint64, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "sur_param_count": ([vp], ctypes.c_int64),
        "sur_param_offsets": ([vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sur_set_params": ([vp, dp], ctypes.c_int),
        "sur_get_params": ([vp, dp], ctypes.c_int),
        "sur_forward": ([vp, dp, i64, dp], ctypes.c_int),
        "sur_loss_grad": ([vp, dp, dp, i64, dp, dp], ctypes.c_int),
        "sur_loss": ([vp, dp, dp, i64, dp], ctypes.c_int),
        "sur_adam_step": ([vp, dp, dp, i64, ctypes.c_float], ctypes.c_int),
        "sur_train": ([vp, dp, dp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64, dp], ctypes.c_int),
        "sur_reconstruct": ([dp, dp, dp, i32, i64, i32, dp, vp], ctypes.c_int),
        "sur_pod": ([dp, i64, i64, i32, dp, dp, dp, dp, ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_int32), vp], ctypes.c_int),
        "sur_fit_trust": ([vp, dp, i64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "sur_trust": ([vp, dp, i64, dp], ctypes.c_int),
        "sur_matmul": ([dp, i64, i64, dp, i64, i64, dp, i32, i32, i32, i32, vp], ctypes.c_int),
        "sur_field_stats": ([dp, i32, i32, dp, dp, i64, dp, dp, dp, vp], ctypes.c_int),
        "sur_last_error": ([vp], ctypes.c_char_p),
        "sur_destroy": ([vp], None),
        "ens_set_centerline": ([vp, i32, dp], ctypes.c_int),
        "ens_quantity_device": ([vp, i32, dp], ctypes.c_int),
        "ens_quantity_stats": ([vp, i32, i32, dp, dp, dp, dp], ctypes.c_int),
        "ens_row_stats_device": ([i64, i32, dp, i32, dp, dp, dp, dp, vp], ctypes.c_int),
        "ens_set_probes": ([vp, i32, dp, i32, dp, i32, i64], ctypes.c_int),
        "ens_set_peak": ([vp, i32], ctypes.c_int),
        "ens_set_geometry_update": ([vp, i32], ctypes.c_int),
        "ens_get_probes": ([vp, dp, dp, dp, ctypes.POINTER(i64)], ctypes.c_int),
        "gmrf_create": ([i32, i32, dp, dp, ctypes.c_double, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "gmrf_sample": ([vp, i32, dp, dp, ctypes.c_double, ctypes.c_double, i32, ctypes.c_double, i32],
                        ctypes.c_int),
        "gmrf_info": ([vp, ctypes.POINTER(gmrf_info_t)], ctypes.c_int),
        "gmrf_last_error": ([vp], ctypes.c_char_p),
        "gmrf_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L
