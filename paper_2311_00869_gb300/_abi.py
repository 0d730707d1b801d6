"""ctypes declarations of the C ABI in include/signedbal.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
i32, i64, u32, u64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class CloudEntry(ctypes.Structure):
    _fields_ = [("hash", u64), ("S", i32), ("count", i32), ("first_tree", i64)]


SIGNATURES = {
    "sb_create": (i32, [ctypes.POINTER(P), ctypes.c_int, P]),
    "sb_destroy": (None, [P]),
    "sb_status_str": (ctypes.c_char_p, [i32]),
    "sb_last_error": (ctypes.c_char_p, [P]),
    "sb_set_allocator": (i32, [P, ALLOC_FN, FREE_FN, P]),
    "sb_sync": (i32, [P]),
    "sb_profile": (i32, [P, ctypes.c_int]),
    "sb_profile_read": (i32, [P, P, P]),
    "sb_stats": (i32, [P, P, i32]),
    "sb_hash_peak": (i32, [P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "sb_set_tuning": (i32, [P, i32, i64]),
    "sb_get_tuning": (i32, [P, i32, P]),
    "sb_load_graph": (i32, [P, i64, i64, P, P, P, u32, ctypes.POINTER(i64), ctypes.POINTER(i64), P]),
    "sb_load_batch": (i32, [P, i64, P, P, P, P, P, u32, P, P]),
    "sb_batch_cloud": (i32, [P, P, P, P]),
    "sb_batch_steps": (i32, [P, u64, i64, i64, i32, i32, P, P]),
    "sb_graph_edges": (i32, [P, P, P, P]),
    "sb_graph_csr": (i32, [P, P, P, P]),
    "sb_sample_trees": (i32, [P, u64, i64, i64, P]),
    "sb_sample_trees_kruskal": (i32, [P, u64, i64, i64, P]),
    "sb_label": (i32, [P, P]),
    "sb_frustration": (i32, [P, P, P]),
    "sb_cloud": (i32, [P, P, i64, ctypes.POINTER(i64), ctypes.POINTER(i32)]),
    "sb_cloud_reset": (i32, [P, i64, i32]),
    "sb_cloud_reset_scalable": (i32, [P, i64]),
    "sb_cloud_state": (i32, [P, i64, P]),
    "sb_cloud_switch": (i32, [P, i64, P, ctypes.POINTER(i64)]),
    "sb_graphL_fwd": (i32, [P, P, i32, P, P]),
    "sb_graphL_bwd": (i32, [P, P, i32, P, P]),
    "sb_graphL_descent": (i32, [P, P, P, i32, f32, i32, i32, P, P, P]),
    "sb_graphL_round": (i32, [P, P, i32, P, P]),
    "sb_graphL_fwd_static": (i32, [P, i64, P, i32, P, P, P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libsignedbal.so; raises if it cannot be built or loaded (there is
    no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libsignedbal.so not built at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(SIGNATURES)
