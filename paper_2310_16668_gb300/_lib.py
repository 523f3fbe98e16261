"""ctypes view of the C-ABI in ``include/skel.h`` (argument marshalling only).

The shared library is built in-tree by ``paper_2310_16668_gb300.build``.
Loading fails loudly when it is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libskel.so")

SKEL_OK = 0
ERRORS = {-1: "SKEL_ERR_ARG", -2: "SKEL_ERR_OOM", -3: "SKEL_ERR_CUDA", -4: "SKEL_ERR_TIMEOUT",
          -5: "SKEL_ERR_NUMERIC", -6: "SKEL_ERR_STATE"}
KERNELS = {"laplace2d": 0, "laplace3d": 1, "helmholtz3d": 2, "helmholtz2d": 3}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_tc": 2}

# every symbol include/skel.h declares
SYMBOLS = ("skel_build", "skel_apply", "skel_apply_transpose", "skel_free", "skel_info",
           "skel_last_error", "skel_plan_get_dims", "skel_plan_export", "skel_plan_import",
           "skel_neighbors_export", "skel_set_profiling", "skel_last_timings",
           "skel_device_status", "skel_direct_noalloc", "skel_apply_batch", "skel_autotune",
           "skel_build_batch", "skel_test_withhold_tile", "skel_test_fail_alloc", "skel_merge",
           "skel_test_set_updown")


class SkelKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("kappa", ctypes.c_double)]


class SkelOptions(ctypes.Structure):
    _fields_ = [("proxy_p", ctypes.c_int), ("nrhs_max", ctypes.c_int),
                ("host_only", ctypes.c_int), ("num_threads", ctypes.c_int), ("device_build", ctypes.c_int),
                ("store_tiles", ctypes.c_int), ("store_stages", ctypes.c_int), ("updown_tc", ctypes.c_int)]


class SkelStats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("dim", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64), ("k_max", ctypes.c_int),
                ("n_index", ctypes.c_int64), ("n_T", ctypes.c_int64),
                ("n_colleague", ctypes.c_int64), ("n_coarse", ctypes.c_int64), ("n_fine", ctypes.c_int64),
                ("pairs_direct", ctypes.c_int64), ("pairs_far", ctypes.c_int64),
                ("n_work_items", ctypes.c_int64),
                ("t_tree", ctypes.c_double), ("t_skel", ctypes.c_double), ("t_upload", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("n_tc_items", ctypes.c_int64),
                ("n_tc_tiles", ctypes.c_int64), ("n_mix_items", ctypes.c_int64),
                ("pairs_tc", ctypes.c_int64), ("skel_on_device", ctypes.c_int),
                ("t_id_kernels", ctypes.c_double), ("id_gflop", ctypes.c_double),
                ("stored_tile_bytes", ctypes.c_int64), ("n_proxy", ctypes.c_int),
                ("pairs_stored", ctypes.c_int64), ("store_mode", ctypes.c_int)]


class SkelPlanDims(ctypes.Structure):
    _fields_ = [("n_boxes", ctypes.c_int64), ("n_index", ctypes.c_int64), ("n_T", ctypes.c_int64),
                ("dim", ctypes.c_int), ("is_complex", ctypes.c_int),
                ("center", ctypes.c_double * 3), ("side", ctypes.c_double)]


class SkelTimings(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("launches", ctypes.c_int), ("n_applies", ctypes.c_int),
                ("ms_main", ctypes.c_double), ("main_launches", ctypes.c_int)]


class SkelTuning(ctypes.Structure):
    _fields_ = [("ms_onfly", ctypes.c_double), ("ms_stored", ctypes.c_double), ("stored", ctypes.c_int),
                ("n_updown", ctypes.c_int), ("n_changed", ctypes.c_int),
                ("ms_updown_default", ctypes.c_double), ("ms_updown_tuned", ctypes.c_double),
                ("tc_stages", ctypes.c_int), ("ms_sym", ctypes.c_double), ("tcs_stages", ctypes.c_int)]


class SkelError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libskel.so not built ({LIB_PATH}); run paper_2310_16668_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.skel_build.argtypes = [P, I64, I, SkelKernel, D, I, ctypes.POINTER(SkelOptions), ctypes.POINTER(P)]
    lib.skel_apply.argtypes = [P, P, P, I, I, P]
    lib.skel_apply_transpose.argtypes = [P, P, P, I, I, P]
    lib.skel_free.argtypes = [P]
    lib.skel_free.restype = None
    lib.skel_info.argtypes = [P, ctypes.POINTER(SkelStats)]
    lib.skel_last_error.restype = ctypes.c_char_p
    lib.skel_last_error.argtypes = []
    lib.skel_plan_get_dims.argtypes = [P, ctypes.POINTER(SkelPlanDims)]
    lib.skel_plan_export.argtypes = [P] + [P] * 10
    lib.skel_plan_import.argtypes = [P, I64, I, SkelKernel, P, D, I64] + [P] * 10 + \
        [ctypes.POINTER(SkelOptions), ctypes.POINTER(P)]
    lib.skel_neighbors_export.argtypes = [P, I, P, P]
    lib.skel_set_profiling.argtypes = [P, I]
    lib.skel_last_timings.argtypes = [P, ctypes.POINTER(SkelTimings)]
    lib.skel_device_status.argtypes = [P]
    lib.skel_direct_noalloc.argtypes = [P, I64, I, SkelKernel, P, P, I, P]
    lib.skel_apply_batch.argtypes = [P, I, P, P, I, I, I, P]
    lib.skel_autotune.argtypes = [P, I, I, P, ctypes.POINTER(SkelTuning)]
    lib.skel_build_batch.argtypes = [I, P, P, I, SkelKernel, D, I, ctypes.POINTER(SkelOptions), P]
    lib.skel_test_withhold_tile.argtypes = [P, D]
    lib.skel_test_fail_alloc.argtypes = [I]
    lib.skel_test_set_updown.argtypes = [P, I]
    lib.skel_merge.argtypes = [P, I, ctypes.POINTER(SkelOptions), ctypes.POINTER(P)]
    for name in SYMBOLS:
        if name not in ("skel_free", "skel_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(rc: int) -> None:
    if rc != SKEL_OK:
        raise SkelError(rc, load().skel_last_error().decode())
