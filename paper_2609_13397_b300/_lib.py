"""ctypes declarations of include/conegs.h (argument marshalling only).

Loads the in-tree libconegs.so.  There is no fallback: if the library is
missing or fails to load, importing the package raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libconegs.so")

c_void_p, c_int, c_int64, c_float, c_size_t, c_uint = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                                       ctypes.c_float, ctypes.c_size_t, ctypes.c_uint)

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NOCONVERGE", 5: "ERR_OVERFLOW",
          6: "ERR_STATE", 7: "ERR_BUDGET"}


class Stats(ctypes.Structure):
    _fields_ = [("n_gaussians", ctypes.c_int64), ("n_visible", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tiles_x", ctypes.c_int32),
                ("tiles_y", ctypes.c_int32), ("n_valid_pixels", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
                ("n_launches", ctypes.c_int64), ("n_walked", ctypes.c_int64), ("n_evaluated", ctypes.c_int64), ("ms_preprocess", ctypes.c_float), ("ms_sort", ctypes.c_float),
                ("ms_raster", ctypes.c_float), ("ms_total", ctypes.c_float), ("ms_raster_main", ctypes.c_float),
                ("n_evaluated_flat", ctypes.c_int64), ("n_flat", ctypes.c_int64)]


class ConegsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_13397_b300.build` "
                          "(the renderer has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "conegs_create": ([ctypes.POINTER(P), c_int, c_size_t], c_int),
        "conegs_destroy": ([P], None),
        "conegs_last_error": ([], ctypes.c_char_p),
        "conegs_version": ([], ctypes.c_char_p),
        "conegs_set_scene": ([P, c_int64, P, P, P, P, P, c_int, c_int, P, P], c_int),
        "conegs_view_create": ([P, ctypes.POINTER(P)], c_int),
        "conegs_view_destroy": ([P], None),
        "conegs_set_camera": ([P, c_int, c_int, c_int, P, P, P, c_float, P], c_int),
        "conegs_render": ([P, P, P, c_uint, P], c_int),
        "conegs_render_batch": ([c_int, P, P, P, c_uint, P], c_int),
        "conegs_render_host_batch": ([c_int, P, P, P, c_uint, P], c_int),
        "conegs_render_host_batch_async": ([c_int, P, P, P, c_uint, P], c_int),
        "conegs_view_host_wait": ([P], c_int),
        "conegs_render_host": ([P, P, P, c_uint, P], c_int),
        "conegs_render_count": ([P, c_uint, ctypes.POINTER(c_int64), ctypes.POINTER(c_size_t), P], c_int),
        "conegs_render_backward": ([P, P, P, P, P, P, P, P, P], c_int),
        "conegs_get_stats": ([P, ctypes.POINTER(Stats)], c_int),
        "conegs_compute_floor": ([P, c_int, P, P, P], c_int),
        "conegs_get_rays": ([P, P, P, P, P, P], c_int),
        "conegs_get_tile_table": ([P, P, P], c_int),
        "conegs_get_bin_counts": ([P, P, P, P], c_int),
        "conegs_get_pairs": ([P, P, P, P], c_int),
        "conegs_radix_sort_pairs": ([P, P, P, c_int64, c_int, c_int, P], c_int),
        "conegs_radix_sort_pairs_noalloc": ([P, P, c_int64, c_int, c_int, P], c_int),
        "conegs_measure_fp32_peak": ([c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                                     c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/conegs.h (for the ABI completeness test)."""
    return ["conegs_create", "conegs_destroy", "conegs_last_error", "conegs_version", "conegs_set_scene",
            "conegs_view_create", "conegs_view_destroy", "conegs_set_camera", "conegs_render", "conegs_render_batch",
            "conegs_render_host_batch", "conegs_render_host_batch_async", "conegs_view_host_wait",
            "conegs_render_host", "conegs_render_count",
            "conegs_render_backward", "conegs_get_stats", "conegs_compute_floor", "conegs_get_rays",
            "conegs_get_tile_table", "conegs_get_bin_counts", "conegs_get_pairs", "conegs_radix_sort_pairs",
            "conegs_radix_sort_pairs_noalloc", "conegs_measure_fp32_peak"]


def check(status: int, what: str = ""):
    if status != 0:
        msg = lib().conegs_last_error().decode(errors="replace")
        raise ConegsError(status, f"{what}: {msg}" if what else msg)
