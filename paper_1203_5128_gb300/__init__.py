"""GB300-native shiftable O(1) Gaussian bilateral filter (arXiv:1203.5128).

The filter runs in libbf (hand-written CUDA for sm_103a behind the C ABI of
include/bf.h); this package is its Python binding.  Importing it does not
load the library; the first call does, and fails loudly if it is missing.
"""
from .api import (  # noqa: F401
    Plan,
    bf_backward,
    bf_destroy,
    bf_execute,
    bf_execute_batch,
    bf_execute_host,
    bf_get_device_status,
    bf_get_info,
    bf_get_sets,
    bf_get_timing,
    bf_maxmin,
    bf_test_stall,
    bf_options_init,
    bf_plan,
    bf_set_timing,
    bf_status_string,
    bilateral_filter,
)
from ._native import BfError  # noqa: F401
