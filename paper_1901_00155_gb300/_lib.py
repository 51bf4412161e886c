"""ctypes binding of libdd.so (include/dd.h).  Argument marshalling only:
every step of the search runs in the library's CUDA kernels.  There is no CPU
fallback -- if the library is missing or cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdd.so")

DD_OK, DD_EINVAL, DD_ENOMEM, DD_ENONFINITE, DD_ETIMEOUT, DD_ECUDA, DD_EBUSY, DD_ENOTSUP = range(8)
DD_FP32, DD_TC_FP16, DD_TC_BF16 = 0, 1, 2


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("paa_w", ctypes.c_int32), ("alphabet", ctypes.c_int32),
                ("early_abandon", ctypes.c_int32), ("paa_mode", ctypes.c_int32), ("phase1_max", ctypes.c_int32),
                ("refine_k", ctypes.c_int32), ("local_cols", ctypes.c_int32), ("word_cols", ctypes.c_int32),
                ("shard_count", ctypes.c_int32), ("shard_index", ctypes.c_int32), ("znorm", ctypes.c_int32),
                ("diag", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Result(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int64), ("nn_distance", ctypes.c_double), ("status", ctypes.c_int32),
                ("exact", ctypes.c_int32), ("computed_pairs", ctypes.c_int64), ("candidates", ctypes.c_int64)]


class View(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("N", ctypes.c_int64), ("n", ctypes.c_int32), ("dict_size", ctypes.c_int32),
                ("stats", ctypes.c_void_p), ("P1", ctypes.c_void_p), ("P2", ctypes.c_void_p),
                ("mu_w", ctypes.c_void_p), ("c_w", ctypes.c_void_p), ("code", ctypes.c_void_p),
                ("freq_hist", ctypes.c_void_p), ("order", ctypes.c_void_p), ("word_start", ctypes.c_void_p),
                ("ncand", ctypes.c_void_p), ("t32", ctypes.c_void_p)]


class BoundView(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("precision", ctypes.c_int32), ("beta", ctypes.c_float),
                ("alpha", ctypes.c_void_p), ("gam", ctypes.c_void_p), ("q2", ctypes.c_void_p)]


class OrderView(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("stride", ctypes.c_int64), ("bins", ctypes.c_int32),
                ("sig", ctypes.c_void_p), ("sigpos", ctypes.c_void_p), ("mubin", ctypes.c_void_p),
                ("binstart", ctypes.c_void_p), ("geom", ctypes.c_void_p)]


class Profile(ctypes.Structure):
    _fields_ = [("dist_launches", ctypes.c_int32), ("precision", ctypes.c_int32), ("dist_ms", ctypes.c_double),
                ("computed_pairs", ctypes.c_int64), ("call_ms", ctypes.c_double), ("reserved", ctypes.c_int64 * 4)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("result", Result), ("queue_ms", ctypes.c_double),
                ("service_ms", ctypes.c_double)]


DD_SERIES_DEVICE = 0
DD_SERIES_HOST = 1


class BatchConfig(ctypes.Structure):
    _fields_ = [("seg_cols", ctypes.c_int32), ("settle_min", ctypes.c_int32), ("settle_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class Wave(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rows", ctypes.c_int32), ("items", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("ms", ctypes.c_double)]


WAVE_KINDS = {0: "exhaustive", 1: "local", 2: "band", 3: "cand", 4: "top", 5: "word", 6: "rest", 7: "time", 8: "settle",
              9: "diag"}

_lock = threading.Lock()
_lib = None

# exported symbol -> (argtypes, restype); every function include/dd.h declares
SIGNATURES = {
    "dd_options_default": ([ctypes.POINTER(Options)], None),
    "dd_plan_footprint": ([ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options)], ctypes.c_size_t),
    "dd_plan_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options),
                        ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    "dd_plan_destroy": ([ctypes.c_void_p], None),
    "dd_find_discord": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Result), ctypes.c_void_p], ctypes.c_int),
    "dd_find_discord_async": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_find_discord_host": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Result), ctypes.c_void_p],
                             ctypes.c_int),
    "dd_find_discord_batched": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Options), ctypes.POINTER(Result),
                                 ctypes.c_void_p], ctypes.c_int),
    "dd_nn_profile": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_nn_profile_diag": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                           ctypes.c_int),
    "dd_nn_rows": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                    ctypes.c_void_p], ctypes.c_int),
    "dd_prep": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dd_plan_view": ([ctypes.c_void_p, ctypes.POINTER(View)], ctypes.c_int),
    "dd_plan_bound_view": ([ctypes.c_void_p, ctypes.POINTER(BoundView)], ctypes.c_int),
    "dd_plan_order_view": ([ctypes.c_void_p, ctypes.POINTER(OrderView)], ctypes.c_int),
    "dd_plan_last_launches": ([ctypes.c_void_p], ctypes.c_int64),
    "dd_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "dd_probe_fma_rate": ([ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p], ctypes.c_int),
    "dd_plan_set_profiling": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "dd_plan_get_profile": ([ctypes.c_void_p, ctypes.POINTER(Profile)], ctypes.c_int),
    "dd_plan_set_graph": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "dd_plan_inject": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "dd_find_discords": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Result), ctypes.c_void_p],
                         ctypes.c_int),
    "dd_plan_get_waves": ([ctypes.c_void_p, ctypes.POINTER(Wave), ctypes.c_int32], ctypes.c_int32),
    "dd_nn_profile_static": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
                             ctypes.c_int),
    "dd_engine_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(Options), ctypes.c_int64,
                          ctypes.c_int32], ctypes.c_int),
    "dd_engine_create_budget": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(Options),
                                 ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t], ctypes.c_int),
    "dd_engine_submit": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                          ctypes.c_int32], ctypes.c_int),
    "dd_engine_poll": ([ctypes.c_void_p, ctypes.POINTER(Completion), ctypes.c_int32, ctypes.c_int32], ctypes.c_int32),
    "dd_engine_outstanding": ([ctypes.c_void_p], ctypes.c_int64),
    "dd_engine_destroy": ([ctypes.c_void_p], None),
    "dd_batch_config_default": ([ctypes.POINTER(BatchConfig)], None),
    "dd_batch_footprint": ([ctypes.c_int32, ctypes.c_int64, ctypes.c_int32], ctypes.c_size_t),
    "dd_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                         ctypes.POINTER(Options), ctypes.POINTER(BatchConfig)], ctypes.c_int),
    "dd_batch_search": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(Result),
                         ctypes.c_void_p], ctypes.c_int),
    "dd_batch_graph_replays": ([ctypes.c_void_p], ctypes.c_int64),
    "dd_batch_set_schedule": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BatchConfig)], ctypes.c_int),
    "dd_batch_destroy": ([ctypes.c_void_p], None),
}


def load(build_if_missing: bool = True):
    """Load libdd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdd.so not found at {LIB_PATH}; build it with python -m paper_1901_00155_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib
