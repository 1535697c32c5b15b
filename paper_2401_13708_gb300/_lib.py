"""ctypes declarations of libhts (include/hts.h).

The library is built in-tree (paper_2401_13708_gb300/_build/libhts.so) by
build.py.  There is no fallback: if the library is missing or cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhts.so")

HTS_OK = 0
ERRORS = {
    -1: "HTS_EINVAL",
    -2: "HTS_ESHAPE",
    -3: "HTS_ENOTSET",
    -4: "HTS_EDOMAIN",
    -5: "HTS_ECUDA",
    -6: "HTS_EOOM",
    -7: "HTS_ENUMERIC",
    -8: "HTS_ETOOLARGE",
    -9: "HTS_ETIMEOUT",
}
NOALLOC_MAX_N = 65536
FP64, FP32_MIXED = 0, 1
EQUAL_LENGTH, EQUAL_AREA = 0, 1
EXACT_KL, PAPER_EQ = 0, 1
HOST, DEVICE = 0, 1
F32, F64 = 0, 1
TREE_LEVELS = 29

EXPORTS = [
    "hts_default_config", "hts_create", "hts_destroy", "hts_set_P", "hts_set_Y", "hts_step", "hts_get_Y",
    "hts_grad", "hts_kl", "hts_last_error", "hts_get_keys", "hts_get_tree", "hts_get_counters",
    "hts_set_counters", "hts_get_state", "hts_set_state", "hts_get_sizes", "hts_set_profiling",
    "hts_get_profile", "hts_exact_grad_noalloc", "hts_set_cosne", "hts_set_segments", "hts_get_segment_Z",
    "hts_kl_segments", "hts_set_graphs", "hts_autotune", "hts_set_tuning", "hts_get_tuning",
    "hts_measure_peaks", "hts_set_walk_split", "hts_update_Y", "hts_get_walk_split", "hts_get_criterion_count",
    "hts_set_wait_test",
]
MAX_SEGMENTS = 64


class HtsConfig(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("split_rule", C.c_int),
        ("grad_form", C.c_int),
        ("metric_pow", C.c_int),
        ("eps", C.c_double),
        ("use_gains", C.c_int),
        ("device", C.c_int),
        ("stream", C.c_void_p),
    ]


class HtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libhts.so and declare its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"libhts.so not found at {path}: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        lib = C.CDLL(path)
        vp, i32, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "hts_default_config": (None, [C.POINTER(HtsConfig)]),
            "hts_create": (i32, [C.POINTER(vp), C.POINTER(HtsConfig)]),
            "hts_destroy": (None, [vp]),
            "hts_set_P": (i32, [vp, i64, i64, vp, vp, vp, i32, i32]),
            "hts_set_Y": (i32, [vp, i64, vp, i32]),
            "hts_step": (i32, [vp, i32, d, d, d, d]),
            "hts_get_Y": (i32, [vp, vp, i32]),
            "hts_grad": (i32, [vp, d, d, vp, vp, i32]),
            "hts_kl": (i32, [vp, d, vp]),
            "hts_last_error": (C.c_char_p, [vp]),
            "hts_get_keys": (i32, [vp, vp, vp, i32]),
            "hts_get_tree": (i32, [vp, i64, vp, vp, vp, vp, vp, vp, vp]),
            "hts_get_counters": (i32, [vp, vp]),
            "hts_set_counters": (i32, [vp, i32]),
            "hts_get_state": (i32, [vp, vp, vp, vp, i32]),
            "hts_set_state": (i32, [vp, vp, vp, i64, i32]),
            "hts_get_sizes": (i32, [vp, vp, vp]),
            "hts_set_profiling": (i32, [vp, i32]),
            "hts_get_profile": (i32, [vp, vp, vp]),
            "hts_exact_grad_noalloc": (i32, [i64, i64, vp, vp, vp, vp, d, i32, vp, vp, vp]),
            "hts_set_cosne": (i32, [vp, d, d, vp, i32]),
            "hts_set_segments": (i32, [vp, i32, vp, vp]),
            "hts_get_segment_Z": (i32, [vp, vp]),
            "hts_kl_segments": (i32, [vp, d, vp]),
            "hts_set_graphs": (i32, [vp, i32]),
            "hts_autotune": (i32, [vp, d, i32, vp]),
            "hts_set_tuning": (i32, [vp, i32, i32]),
            "hts_get_tuning": (i32, [vp, vp]),
            "hts_measure_peaks": (i32, [i32, vp]),
            "hts_set_walk_split": (i32, [vp, i32]),
            "hts_update_Y": (i32, [vp, vp, i32]),
            "hts_get_walk_split": (i32, [vp, vp]),
            "hts_get_criterion_count": (i32, [vp, vp]),
            "hts_set_wait_test": (i32, [vp, i32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(lib, ctx, code: int):
    if code != HTS_OK:
        msg = lib.hts_last_error(ctx)
        raise HtsError(code, msg.decode() if msg else "")
    return code
