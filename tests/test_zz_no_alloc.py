"""GPU test of bf_execute_noalloc, the entry point for callers that cannot
allocate device memory while they run (a pipeline that reserves all of its
GPU memory at start-up, or an application that only lends this library its
image buffers).  It keeps its scratch in a fixed static device array instead
of a plan's workspace.

Its output must match the plan-based bf_execute (same algorithm: global T,
Algorithm 2 truncation, FP32 planes, no FP32 recheck -- the allocation-free
entry point has none) within the forward tolerance of the other GPU tests,
on two calls in a row -- the second call reuses the static
array the first one left behind, so it also checks that the scratch is
cleared where it must start at zero.  The file is named to be collected
last, so a run that stops at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu

TOL8 = 1e-3   # gray levels, as the forward parity tests


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build, _native
    build.build()
    return _native.lib()


def noalloc(lib, f, out, sigma_s, sigma_r, eps, value_range=255.0):
    import torch
    from paper_1203_5128_gb300 import _native as nat
    code = lib.bf_execute_noalloc(f.data_ptr(), f.stride(0), out.data_ptr(), out.stride(0),
                                  f.shape[0], f.shape[1], sigma_s, sigma_r, eps,
                                  ctypes.c_float(value_range),
                                  torch.cuda.current_stream().cuda_stream)
    assert code == nat.BF_OK, lib.bf_status_string(code)


def device_status(lib):
    import torch
    bits = ctypes.c_uint()
    lib.bf_noalloc_device_status(torch.cuda.current_stream().cuda_stream, ctypes.byref(bits))
    return bits.value


def test_noalloc_matches_plan_path_on_two_calls(lib):
    import torch
    import paper_1203_5128_gb300 as bf
    # radii 9 and 15 (tall tiles), 30 and 48 (the fused kernel's small tiles:
    # there is no two-pass workspace), ragged sizes
    cases = [(300, 257, 3.0, 20.0, 0.01, 11), (256, 320, 5.0, 10.0, 0.01, 12),
             (97, 203, 10.0, 20.0, 0.01, 13), (65, 97, 16.0, 25.0, 0.01, 14)]
    for H, W, ss, sr, eps, seed in cases:
        f = torch.from_numpy(synth.g8(H, W, seed=seed)).cuda()
        ref = bf.bf_execute(bf.bf_plan(H, W, ss, sr, eps, t_mode="global", trunc_rule="alg2",
                                       fp32_recheck=0.0), f)
        out = torch.full_like(f, float("nan"))
        noalloc(lib, f, out, ss, sr, eps)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert np.isfinite(err) and err <= TOL8, "max-abs %.3g gray levels" % err
        assert device_status(lib) == 0


def test_noalloc_reports_order_overflow(lib):
    """Pixels outside [0, value_range] can need an order above the static
    table: the output is then a copy of the input, the call still returns
    BF_OK, and the status bit is read (and cleared) by
    bf_noalloc_device_status."""
    import torch
    from paper_1203_5128_gb300 import _native as nat
    f_np = synth.g8(64, 96, seed=21)
    f_np[10:20, 10:20] = 2000.0           # far above value_range = 255
    f = torch.from_numpy(f_np).cuda()
    out = torch.full_like(f, float("nan"))
    noalloc(lib, f, out, 2.0, 10.0, 0.01)
    torch.cuda.synchronize()
    assert torch.equal(out, f)
    bits = ctypes.c_uint()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.bf_noalloc_device_status(s, ctypes.byref(bits)) == nat.BF_ERR_DEVICE_STATUS
    assert bits.value & nat.BF_DEV_ORDER_TOO_LARGE
    assert lib.bf_noalloc_device_status(s, ctypes.byref(bits)) == nat.BF_OK and bits.value == 0


def test_noalloc_rejects_sizes_above_its_scratch(lib):
    import torch
    from paper_1203_5128_gb300 import _native as nat
    f = torch.zeros((64, 64), device="cuda")
    out = torch.empty_like(f)
    s = torch.cuda.current_stream().cuda_stream
    # R = ceil(3 * 17) = 51 > 48
    assert lib.bf_execute_noalloc(f.data_ptr(), 64, out.data_ptr(), 64, 64, 64, 17.0, 20.0,
                                  0.01, ctypes.c_float(255.0), s) == nat.BF_ERR_NOT_SUPPORTED
    # order for [0, 255] at sigma_r = 2 is 6589 > 1024
    assert lib.bf_execute_noalloc(f.data_ptr(), 64, out.data_ptr(), 64, 64, 64, 2.0, 2.0,
                                  0.01, ctypes.c_float(255.0), s) == nat.BF_ERR_ORDER_TOO_LARGE
    assert lib.bf_execute_noalloc(None, 64, out.data_ptr(), 64, 64, 64, 2.0, 20.0,
                                  0.01, ctypes.c_float(255.0), s) == nat.BF_ERR_INVALID_ARG
