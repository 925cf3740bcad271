"""GB300 explicit ensemble solver for the segregated vessel-wall model
(Li & Schiavazzi, arXiv 2101.09059): C ABI in include/ens.h, CUDA kernels in csrc/,
and a thin Python binding."""
from ._lib import build, load, declared_functions
from .fields import FieldSampler
from .ensemble import (Ensemble, Batch, EnsError, FP64, FP32_FORCE, KAHAN32, PRECISIONS, BATCH_AUTO,
                       BATCH_GRAPH, BATCH_PERSISTENT, BATCH_SEQUENCE)

__all__ = ["build", "load", "declared_functions", "FieldSampler", "Ensemble", "Batch", "EnsError", "BATCH_AUTO",
           "BATCH_GRAPH", "BATCH_PERSISTENT", "BATCH_SEQUENCE", "FP64", "FP32_FORCE",
           "KAHAN32", "PRECISIONS"]
