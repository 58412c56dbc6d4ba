"""ctypes declarations of libbf (include/bf.h).  Marshalling only.

Loading fails loudly when the library has not been built: there is no
fallback path of any kind.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbf.so")

# status codes (bf_status)
BF_OK = 0
BF_ERR_INVALID_ARG = 1
BF_ERR_ORDER_TOO_LARGE = 2
BF_ERR_ALLOC = 3
BF_ERR_CUDA = 4
BF_ERR_TIMEOUT = 5
BF_ERR_NO_FORWARD = 6
BF_ERR_NOT_SUPPORTED = 7
BF_ERR_DEVICE_STATUS = 8

BF_T_FIXED, BF_T_GLOBAL, BF_T_TILE = 0, 1, 2
BF_RULE_ALG2, BF_RULE_TRUNC, BF_RULE_CHERNOFF = 0, 1, 2
BF_FILTER_AUTO, BF_FILTER_FIR, BF_FILTER_YVV = 0, 1, 2
BF_PLANES_FP32, BF_PLANES_BF16, BF_PLANES_FP16 = 0, 1, 2
BF_SPATIAL_GAUSS, BF_SPATIAL_BOX = 0, 1
BF_RANGE_COSINE, BF_RANGE_POLY = 0, 1
BF_DEV_ORDER_TOO_LARGE, BF_DEV_TIMEOUT, BF_DEV_BAD_WORK = 1, 2, 4


class bf_options(ctypes.Structure):
    _fields_ = [
        ("t_mode", ctypes.c_int),
        ("t_fixed", ctypes.c_float),
        ("value_range", ctypes.c_float),
        ("trunc_rule", ctypes.c_int),
        ("filter", ctypes.c_int),
        ("plane_dtype", ctypes.c_int),
        ("n_max", ctypes.c_int),
        ("t_tile", ctypes.c_int),
        ("spin_limit", ctypes.c_longlong),
        ("spatial", ctypes.c_int),
        ("lowp_recheck", ctypes.c_float),
        ("range_kernel", ctypes.c_int),
        ("patch_mask", ctypes.c_int),
        ("fp32_recheck", ctypes.c_float),
        ("reserved", ctypes.c_int * 3),
    ]


class bf_info(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int), ("W", ctypes.c_int), ("R", ctypes.c_int),
        ("n_sets", ctypes.c_int),
        ("T", ctypes.c_float),
        ("N", ctypes.c_int), ("M", ctypes.c_int), ("K", ctypes.c_int),
        ("n_guarded", ctypes.c_longlong),
        ("terms_total", ctypes.c_longlong),
        ("device_status", ctypes.c_uint),
        ("filter", ctypes.c_int), ("plane_dtype", ctypes.c_int), ("t_mode", ctypes.c_int),
        ("tile_h", ctypes.c_int), ("tile_w", ctypes.c_int),
        ("n_rechecked", ctypes.c_longlong),
    ]


# every symbol include/bf.h declares, with its prototype
_P, _I, _D, _Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_PP = ctypes.POINTER(ctypes.c_void_p)
PROTOTYPES = {
    "bf_options_init": (None, [ctypes.POINTER(bf_options)]),
    "bf_plan": (_I, [_I, _I, _D, _D, _D, ctypes.POINTER(bf_options), _PP]),
    "bf_execute": (_I, [_P, _P, _Z, _P, _Z, _P]),
    "bf_execute_host": (_I, [_P, _P, _P, _P]),
    "bf_backward": (_I, [_P, _P, _P, _P, _Z, _P]),
    "bf_execute_batch": (_I, [_I, _P, _P, _P, _P]),
    "bf_get_info": (_I, [_P, ctypes.POINTER(bf_info)]),
    "bf_get_sets": (_I, [_P, _P, _P, _P, _I]),
    "bf_get_device_status": (_I, [_P, ctypes.POINTER(ctypes.c_uint)]),
    "bf_destroy": (None, [_P]),
    "bf_status_string": (ctypes.c_char_p, [_I]),
    "bf_maxmin": (_I, [_P, _I, _I, _Z, _I, _P, _P, _P]),
    "bf_test_stall": (_I, [_P, _I]),
    "bf_set_timing": (_I, [_P, _I]),
    "bf_execute_noalloc": (_I, [_P, _Z, _P, _Z, _I, _I, _D, _D, _D, ctypes.c_float, _P]),
    "bf_noalloc_device_status": (_I, [_P, ctypes.POINTER(ctypes.c_uint)]),
    "bf_get_timing": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I)]),
}

_lib = None


class BfError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().bf_status_string(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (status %d)" % (what, msg, code))


def lib():
    """The loaded libbf (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libbf.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
            "g.build()\"` or `python paper_1203_5128_gb300/build.py`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code: int, what: str):
    if code != BF_OK:
        raise BfError(code, what)
