"""ctypes loader for libraster.so: argument marshalling only.

The library is built in-tree by ``paper_1907_03620_gb300.build``.  There is no
CPU fallback: if the shared library is missing or fails to load, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import builder as _build

_lock = threading.Lock()
_lib = None

OK = 0
E_ARG, E_RANGE, E_OOM, E_TABLE_FULL, E_CUDA, E_INTERNAL, E_STATE, E_LIMIT = 1, 2, 3, 4, 5, 6, 7, 8
STATIC_MAX_POINTS = 524288
NOISE = -(2 ** 63)
INVALID_KEY = -(2 ** 63) + 1  # tile key of a point that did not project (RASTER_INVALID_KEY)
CHEBYSHEV, MANHATTAN, MAX_DELTA = 0, 1, 4  # RASTER_CHEBYSHEV, RASTER_MANHATTAN, RASTER_MAX_DELTA
NAMES = {0: "RASTER_OK", 1: "RASTER_E_ARG", 2: "RASTER_E_RANGE", 3: "RASTER_E_OOM", 4: "RASTER_E_TABLE_FULL",
         5: "RASTER_E_CUDA", 6: "RASTER_E_INTERNAL", 7: "RASTER_E_STATE", 8: "RASTER_E_LIMIT"}


class RasterError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().raster_strerror(status).decode() if _lib is not None else ""
        super().__init__(f"{where}: {NAMES.get(status, status)} ({msg})")


class Params(ctypes.Structure):
    """raster_params"""
    _fields_ = [("precision", ctypes.c_double), ("tau", ctypes.c_uint32), ("mu", ctypes.c_uint32),
                ("metric", ctypes.c_uint32), ("delta", ctypes.c_uint32), ("groups", ctypes.c_uint32),
                ("dims", ctypes.c_uint32)]


class TableStats(ctypes.Structure):
    """raster_table_stats_t"""
    _fields_ = [("capacity", ctypes.c_int64), ("occupied", ctypes.c_int64), ("probe_sum", ctypes.c_int64),
                ("probe_max", ctypes.c_int64)]


class Instance(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("n", ctypes.c_int64), ("precision", ctypes.c_double),
                ("tau", ctypes.c_uint32), ("mu", ctypes.c_uint32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("load", ctypes.c_double), ("block", ctypes.c_int32), ("width", ctypes.c_int32),
                ("preagg", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("table_slots", ctypes.c_int64), ("result_rows", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("reserve_bytes", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("steps", "points", "waiting", "active", "completed_unpolled",
                                              "table_slots_used", "result_rows_used", "device_bytes",
                                              "refused", "gpu_us")]


class Clusters(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("count", ctypes.c_void_p), ("cid", ctypes.c_void_p),
                ("n_tiles", ctypes.c_int64), ("n_clusters", ctypes.c_int64), ("n_distinct", ctypes.c_int64),
                ("n_significant", ctypes.c_int64), ("n_points", ctypes.c_int64)]


def header_functions() -> list[str]:
    """Names of the functions declared in include/*.h (for export checks)."""
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    names = []
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(raster_[a-z0-9_]+)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def _declare(L):
    vp, i64, u32, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
    sig = {
        "raster_create": (ci, [dbl, u32, u32, ctypes.POINTER(vp)]),
        "raster_create_ex": (ci, [ctypes.POINTER(Params), ctypes.POINTER(vp)]),
        "raster_reserve": (ci, [vp, i64]),
        "raster_contract": (ci, [vp, vp, i64, vp]),
        "raster_contract_keys": (ci, [vp, vp, i64, vp, vp]),
        "raster_key_labels": (ci, [vp, vp, i64, vp, vp]),
        "raster_contract_host": (ci, [vp, vp, i64, vp]),
        "raster_agglomerate": (ci, [vp, ctypes.POINTER(Clusters)]),
        "raster_contract_tiles": (ci, [vp, vp, vp, i64, vp]),
        "raster_point_labels": (ci, [vp, vp, i64, vp, vp]),
        "raster_point_labels_host": (ci, [vp, vp, i64, vp, vp]),
        "raster_cluster_host": (ci, [vp, vp, i64, vp, ctypes.POINTER(Clusters), vp]),
        "raster_table_stats": (ci, [vp, ctypes.POINTER(TableStats)]),
        "raster_export_tiles": (ci, [vp, vp, vp, i64, ctypes.POINTER(i64)]),
        "raster_point_groups": (ci, [vp, vp, i64, vp, vp, i64, ctypes.POINTER(i64), vp]),
        "raster_reset": (ci, [vp, vp]),
        "raster_status": (ci, [vp]),
        "raster_get_scale": (dbl, [vp]),
        "raster_table_capacity": (i64, [vp]),
        "raster_destroy": (ci, [vp]),
        "raster_kernel_launches": (ctypes.c_uint64, []),
        "raster_set_test_limits": (ci, [ctypes.c_int32, ctypes.c_int32]),
        "raster_count_tiles_static": (ci, [vp, i64, dbl, vp, vp, ctypes.POINTER(i64), vp]),
        "raster_strerror": (ctypes.c_char_p, [ci]),
        "raster_batch_create": (ci, [ctypes.POINTER(Instance), ctypes.c_int32, ctypes.POINTER(BatchConfig),
                                     ctypes.POINTER(vp)]),
        "raster_batch_run": (ci, [vp, vp]),
        "raster_batch_wait": (ci, [vp]),
        "raster_batch_result": (ci, [vp, ctypes.c_int32, ctypes.POINTER(Clusters)]),
        "raster_batch_device_bytes": (i64, [vp]),
        "raster_batch_destroy": (ci, [vp]),
        "raster_server_create": (ci, [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]),
        "raster_server_submit": (ci, [vp, i64, dbl, u32, u32, i64, ctypes.c_int32]),
        "raster_server_push": (ci, [vp, i64, vp, i64]),
        "raster_server_poll": (ci, [vp, ctypes.c_int32, ctypes.POINTER(i64), ctypes.POINTER(Clusters),
                                    ctypes.POINTER(dbl)]),
        "raster_server_release": (ci, [vp, i64]),
        "raster_server_stats": (ci, [vp, ctypes.POINTER(ServerStats)]),
        "raster_server_destroy": (ci, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def lib():
    """Load (building first if needed) the native library; raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def check(status: int, where: str):
    if status != OK:
        raise RasterError(status, where)
