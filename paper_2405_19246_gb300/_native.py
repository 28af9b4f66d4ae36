"""ctypes binding of the C ABI declared in ``include/mmot.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libmmot_gb300.so``.  There is no fallback: if the library is missing
or cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmot_gb300.so")

MMOT_OK = 0
STATUS_NAMES = {
    0: "MMOT_OK", 1: "MMOT_ERR_INVALID_ARG", 2: "MMOT_ERR_UNSORTED", 3: "MMOT_ERR_OOM",
    4: "MMOT_ERR_CUDA", 5: "MMOT_ERR_TIMEOUT", 6: "MMOT_ERR_NOT_CONVERGED",
    7: "MMOT_ERR_NONFINITE", 8: "MMOT_ERR_RANGE",
}
MMOT_FP64 = 0
MMOT_FP32_SCAN_FP64_POT = 1
MMOT_OPT_CHECK_EVERY = 1
MMOT_OPT_SPIN_LIMIT = 2
MMOT_OPT_USE_GRAPH = 3
MMOT_OPT_PROFILE = 4
MMOT_OPT_TEST_HOLD = 5

# every symbol include/mmot.h declares
EXPORTED = [
    "mmot_plan_create", "mmot_marginal", "mmot_sinkhorn_step", "mmot_solve", "mmot_objective",
    "mmot_get_potentials", "mmot_set_potentials", "mmot_reset_potentials", "mmot_set_option",
    "mmot_get_profile", "mmot_get_info", "mmot_set_memory_limit", "mmot_memory_in_use", "mmot_marginal_noalloc",
    "mmot_shard_create", "mmot_shard_operator", "mmot_shard_set_inflow", "mmot_shard_update", "mmot_shard_residual",
    "mmot_ftvp2d",
    "mmot_batch_create", "mmot_batch_step", "mmot_batch_reset", "mmot_batch_solve", "mmot_batch_freeze", "mmot_batch_status",
    "mmot_batch_get_potentials", "mmot_batch_set_potentials", "mmot_batch_get_info", "mmot_batch_destroy",
    "mmot_destroy", "mmot_last_error",
]


class MmotResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("residual", ctypes.c_double), ("W", ctypes.c_double),
                ("primal", ctypes.c_double), ("dual", ctypes.c_double), ("mass", ctypes.c_double)]


class MmotPlanInfo(ctypes.Structure):
    _fields_ = [("total_points", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("tile_points", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("launches_per_iteration", ctypes.c_int), ("precision", ctypes.c_int),
                ("kernel_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("uniform_grid", ctypes.c_int)]


class MmotBatchInfo(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("groups", ctypes.c_int), ("total_points", ctypes.c_int64),
                ("tiles", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


class MmotError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmmot_gb300.so not built: run __graft_entry__.build() "
                               "or python -m paper_2405_19246_gb300._build")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.mmot_plan_create.argtypes = [i, P(i64), P(vp), P(vp), d, i, i, vp, P(vp)]
        L.mmot_marginal.argtypes = [vp, i, i, vp]
        L.mmot_sinkhorn_step.argtypes = [vp, i, P(d)]
        L.mmot_solve.argtypes = [vp, d, i, P(MmotResult)]
        L.mmot_objective.argtypes = [vp, P(MmotResult)]
        L.mmot_get_potentials.argtypes = [vp, i, vp]
        L.mmot_set_potentials.argtypes = [vp, i, vp]
        L.mmot_reset_potentials.argtypes = [vp]
        L.mmot_set_option.argtypes = [vp, i, i64]
        L.mmot_get_profile.argtypes = [vp, i, P(i64), P(d), i]
        L.mmot_get_info.argtypes = [vp, P(MmotPlanInfo)]
        L.mmot_set_memory_limit.argtypes = [i64]
        L.mmot_memory_in_use.argtypes = [ctypes.POINTER(i64)]
        L.mmot_marginal_noalloc.argtypes = [i, P(i64), P(vp), P(vp), d, i, i, vp, vp]
        L.mmot_shard_create.argtypes = [i, P(i64), P(vp), P(vp), P(i64), d, i, i, vp, P(vp)]
        L.mmot_shard_operator.argtypes = [vp, i, vp]
        L.mmot_shard_set_inflow.argtypes = [vp, i, vp, vp]
        L.mmot_shard_update.argtypes = [vp, i]
        L.mmot_shard_residual.argtypes = [vp, i, P(d)]
        L.mmot_ftvp2d.argtypes = [i64, i64, vp, vp, d, d, vp, vp]
        L.mmot_batch_create.argtypes = [i, P(i), P(i64), P(vp), P(vp), P(d), i, i, vp, P(vp)]
        L.mmot_batch_step.argtypes = [vp, i, d, P(i)]
        L.mmot_batch_reset.argtypes = [vp]
        L.mmot_batch_solve.argtypes = [vp, d, i, i, P(MmotResult)]
        L.mmot_batch_freeze.argtypes = [vp, i]
        L.mmot_batch_status.argtypes = [vp, i, P(i), P(d), P(i)]
        L.mmot_batch_get_potentials.argtypes = [vp, i, i, vp]
        L.mmot_batch_set_potentials.argtypes = [vp, i, i, vp]
        L.mmot_batch_get_info.argtypes = [vp, P(MmotBatchInfo)]
        L.mmot_batch_destroy.argtypes = [vp]
        L.mmot_destroy.argtypes = [vp]
        L.mmot_destroy.restype = None
        L.mmot_last_error.argtypes = []
        L.mmot_last_error.restype = ctypes.c_char_p
        for name in EXPORTED[:-2]:
            getattr(L, name).restype = ctypes.c_int
        L.mmot_batch_destroy.restype = None
        _lib = L
    return _lib


def check(status):
    if status != MMOT_OK:
        raise MmotError(status, lib().mmot_last_error().decode())
    return status
