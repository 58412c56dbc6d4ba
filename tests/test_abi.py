"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/bf.h declares, and rejects bad arguments before it touches
the device."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "bf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1203_5128_gb300 import build, _native
    build.build()
    return _native.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["bf_plan", "bf_execute", "bf_backward", "bf_execute_batch", "bf_get_info",
                 "bf_get_device_status", "bf_destroy", "bf_status_string", "bf_execute_host",
                 "bf_maxmin", "bf_options_init", "bf_get_sets"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1203_5128_gb300 import _native
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _native.PROTOTYPES, name


def test_status_strings(lib):
    for code in range(0, 9):
        s = lib.bf_status_string(code)
        assert s and s != b"unknown status"
    assert lib.bf_status_string(99) == b"unknown status"


def test_options_defaults(lib):
    from paper_1203_5128_gb300 import _native as nat
    o = nat.bf_options()
    lib.bf_options_init(ctypes.byref(o))
    assert o.t_mode == nat.BF_T_GLOBAL and o.value_range == 255.0
    assert o.trunc_rule == nat.BF_RULE_ALG2 and o.n_max == 4096 and o.t_tile == 64
    assert o.plane_dtype == nat.BF_PLANES_FP32 and o.spatial == nat.BF_SPATIAL_GAUSS
    assert abs(o.lowp_recheck - 0.05) < 1e-7 and abs(o.fp32_recheck - 0.05) < 1e-7
    # the struct has the size the header gives it (reserved words included)
    assert ctypes.sizeof(nat.bf_options) == 4 * 8 + 8 + 4 + 4 + 4 * 6


@pytest.mark.parametrize("args", [
    (0, 10, 1.0, 10.0, 0.0),      # empty image
    (10, 0, 1.0, 10.0, 0.0),
    (10, 10, 0.0, 10.0, 0.0),     # sigma_s must be > 0
    (10, 10, 1.0, -1.0, 0.0),     # sigma_r must be > 0
    (10, 10, 1.0, 10.0, 1.0),     # eps in [0, 1)
    (10, 10, 1.0, 10.0, -0.1),
    (10, 10, float("nan"), 10.0, 0.0),
])
def test_plan_rejects_bad_arguments(lib, args):
    from paper_1203_5128_gb300 import _native as nat
    h = ctypes.c_void_p()
    assert lib.bf_plan(*args, None, ctypes.byref(h)) == nat.BF_ERR_INVALID_ARG
    assert not h.value


def test_plan_rejects_bad_options(lib):
    from paper_1203_5128_gb300 import _native as nat
    h = ctypes.c_void_p()
    for field, val, code in [("t_mode", 7, nat.BF_ERR_INVALID_ARG),
                             ("trunc_rule", 5, nat.BF_ERR_INVALID_ARG),
                             ("value_range", 0.0, nat.BF_ERR_INVALID_ARG),
                             ("n_max", 0, nat.BF_ERR_INVALID_ARG),
                             ("lowp_recheck", -0.1, nat.BF_ERR_INVALID_ARG),
                             ("lowp_recheck", 1.0, nat.BF_ERR_INVALID_ARG),
                             ("fp32_recheck", -0.1, nat.BF_ERR_INVALID_ARG),
                             ("fp32_recheck", 1.0, nat.BF_ERR_INVALID_ARG),
                             ("n_max", 100000, nat.BF_ERR_NOT_SUPPORTED)]:
        o = nat.bf_options()
        lib.bf_options_init(ctypes.byref(o))
        setattr(o, field, val)
        assert lib.bf_plan(64, 64, 1.0, 10.0, 0.0, ctypes.byref(o), ctypes.byref(h)) == code
    o = nat.bf_options()
    lib.bf_options_init(ctypes.byref(o))
    o.t_mode = nat.BF_T_TILE
    o.t_tile = 48                              # must be a multiple of 64
    assert lib.bf_plan(64, 64, 1.0, 10.0, 0.0, ctypes.byref(o), ctypes.byref(h)) == \
        nat.BF_ERR_INVALID_ARG
    o.reserved[2] = 1
    o.t_tile = 64
    assert lib.bf_plan(64, 64, 1.0, 10.0, 0.0, ctypes.byref(o), ctypes.byref(h)) == \
        nat.BF_ERR_INVALID_ARG


def test_plan_rejects_bad_box_options(lib):
    """The box filter of Sec. 4 takes sigma_s as its radius: a whole number
    >= 1.  It has no recursive form, and unknown spatial kinds are errors."""
    from paper_1203_5128_gb300 import _native as nat
    h = ctypes.c_void_p()
    for sigma_s, spatial, filt, code in [(2.5, nat.BF_SPATIAL_BOX, nat.BF_FILTER_AUTO,
                                          nat.BF_ERR_INVALID_ARG),
                                         (0.5, nat.BF_SPATIAL_BOX, nat.BF_FILTER_FIR,
                                          nat.BF_ERR_INVALID_ARG),
                                         (3.0, nat.BF_SPATIAL_BOX, nat.BF_FILTER_YVV,
                                          nat.BF_ERR_NOT_SUPPORTED),
                                         (3.0, 2, nat.BF_FILTER_AUTO, nat.BF_ERR_INVALID_ARG),
                                         (3.0, -1, nat.BF_FILTER_AUTO, nat.BF_ERR_INVALID_ARG)]:
        o = nat.bf_options()
        lib.bf_options_init(ctypes.byref(o))
        o.spatial = spatial
        o.filter = filt
        assert lib.bf_plan(64, 64, sigma_s, 10.0, 0.0, ctypes.byref(o), ctypes.byref(h)) == code
        assert not h.value


def test_calls_reject_null_plan(lib):
    from paper_1203_5128_gb300 import _native as nat
    assert lib.bf_execute(None, None, 0, None, 0, None) == nat.BF_ERR_INVALID_ARG
    assert lib.bf_backward(None, None, None, None, 0, None) == nat.BF_ERR_INVALID_ARG
    assert lib.bf_get_info(None, None) == nat.BF_ERR_INVALID_ARG
    assert lib.bf_get_device_status(None, None) == nat.BF_ERR_INVALID_ARG
    assert lib.bf_maxmin(None, 4, 4, 4, 1, None, None, None) == nat.BF_ERR_INVALID_ARG
    lib.bf_destroy(None)


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    """No silent fallback: a missing libbf.so is an ImportError."""
    from paper_1203_5128_gb300 import _native as nat
    monkeypatch.setattr(nat, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nat, "_lib", None)
    with pytest.raises(ImportError):
        nat.lib()
