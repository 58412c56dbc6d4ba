"""Python binding of include/bf.h: the same entry points, torch tensors in.

Argument marshalling only: every step of the filter runs in libbf's CUDA
kernels.  Device images are float32 CUDA tensors (2-D, unit column stride);
their row stride is passed as the pitch.  Work goes on the current torch
stream unless a stream is given.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _native as nat

# names of the option enums (strings accepted by bf_plan)
T_MODES = {"fixed": nat.BF_T_FIXED, "global": nat.BF_T_GLOBAL, "tile": nat.BF_T_TILE}
RULES = {"alg2": nat.BF_RULE_ALG2, "trunc": nat.BF_RULE_TRUNC, "chernoff": nat.BF_RULE_CHERNOFF}
FILTERS = {"auto": nat.BF_FILTER_AUTO, "fir": nat.BF_FILTER_FIR, "yvv": nat.BF_FILTER_YVV}
PLANES = {"fp32": nat.BF_PLANES_FP32, "bf16": nat.BF_PLANES_BF16, "fp16": nat.BF_PLANES_FP16}
SPATIALS = {"gauss": nat.BF_SPATIAL_GAUSS, "box": nat.BF_SPATIAL_BOX}
RANGE_KERNELS = {"cosine": nat.BF_RANGE_COSINE, "poly": nat.BF_RANGE_POLY}


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_image(t, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2:
        raise ValueError("%s must be a 2-D float32 CUDA tensor" % name)
    if t.stride(1) != 1:
        raise ValueError("%s must have unit column stride" % name)


def bf_status_string(code: int) -> str:
    return nat.lib().bf_status_string(code).decode()


def bf_options_init(**kw) -> nat.bf_options:
    """bf_options with the library defaults, then keyword overrides
    (t_mode, t_fixed, value_range, trunc_rule, filter, plane_dtype, n_max,
    t_tile, spin_limit, spatial, lowp_recheck, range_kernel, patch_mask, fp32_recheck;
    enum fields accept their lower-case names)."""
    o = nat.bf_options()
    nat.lib().bf_options_init(ctypes.byref(o))
    table = {"t_mode": T_MODES, "trunc_rule": RULES, "filter": FILTERS, "plane_dtype": PLANES,
             "spatial": SPATIALS, "range_kernel": RANGE_KERNELS}
    fields = {name for name, _ in nat.bf_options._fields_ if name != "reserved"}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError("unknown bf_options field %r (known: %s)" % (k, ", ".join(sorted(fields))))
        if v is None:
            continue
        if k in table and isinstance(v, str):
            if v not in table[k]:
                raise ValueError("%s=%r: expected one of %s" % (k, v, ", ".join(sorted(table[k]))))
            v = table[k][v]
        setattr(o, k, v)
    return o


@dataclass
class Info:
    H: int
    W: int
    R: int
    n_sets: int
    T: float
    N: int
    M: int
    K: int
    n_guarded: int
    terms_total: int
    device_status: int
    filter: int
    plane_dtype: int
    t_mode: int
    tile_h: int
    tile_w: int
    n_rechecked: int


class Plan:
    """Owner of a bf_plan_t (bf_destroy on close / garbage collection)."""

    def __init__(self, H: int, W: int, sigma_s: float, sigma_r: float, eps: float = 0.0, **opts):
        self.H, self.W = int(H), int(W)
        self.sigma_s, self.sigma_r, self.eps = float(sigma_s), float(sigma_r), float(eps)
        self.options = bf_options_init(**opts)
        h = ctypes.c_void_p()
        nat.check(nat.lib().bf_plan(self.H, self.W, self.sigma_s, self.sigma_r, self.eps,
                                    ctypes.byref(self.options), ctypes.byref(h)), "bf_plan")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            nat.lib().bf_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def bf_plan(H, W, sigma_s, sigma_r, eps=0.0, **opts) -> Plan:
    return Plan(H, W, sigma_s, sigma_r, eps, **opts)


def bf_execute(plan: Plan, f, out=None, stream=None):
    """Algorithm 2 on a device image; returns out (allocated if None)."""
    import torch
    _check_image(f, "f")
    if f.shape != (plan.H, plan.W):
        raise ValueError("f is %s, plan is %dx%d" % (tuple(f.shape), plan.H, plan.W))
    if out is None:
        out = torch.empty_like(f)
    _check_image(out, "out")
    nat.check(nat.lib().bf_execute(plan.handle, f.data_ptr(), f.stride(0), out.data_ptr(),
                                   out.stride(0), _stream_ptr(stream)), "bf_execute")
    return out


def bf_execute_host(plan: Plan, f_host, out_host=None, stream=None):
    """bf_execute on host (CPU) float32 contiguous tensors; synchronising."""
    import torch
    if f_host.is_cuda or f_host.dtype != torch.float32 or not f_host.is_contiguous():
        raise ValueError("f_host must be a contiguous float32 CPU tensor")
    if out_host is None:
        out_host = torch.empty_like(f_host)
    nat.check(nat.lib().bf_execute_host(plan.handle, f_host.data_ptr(), out_host.data_ptr(),
                                        _stream_ptr(stream)), "bf_execute_host")
    return out_host


def bf_backward(plan: Plan, f, grad_out, grad_in=None, stream=None):
    import torch
    _check_image(f, "f")
    _check_image(grad_out, "grad_out")
    if grad_in is None:
        grad_in = torch.empty_like(f)
    _check_image(grad_in, "grad_in")
    if not (f.stride(0) == grad_out.stride(0) == grad_in.stride(0)):
        raise ValueError("f, grad_out and grad_in must share a row pitch")
    nat.check(nat.lib().bf_backward(plan.handle, f.data_ptr(), grad_out.data_ptr(),
                                    grad_in.data_ptr(), f.stride(0), _stream_ptr(stream)),
              "bf_backward")
    return grad_in


def bf_execute_batch(plans, fs, outs=None, stream=None):
    import torch
    n = len(plans)
    if outs is None:
        outs = [torch.empty_like(f) for f in fs]
    for f, o, p in zip(fs, outs, plans):
        _check_image(f, "f")
        _check_image(o, "out")
        if not (f.is_contiguous() and o.is_contiguous()) or f.shape != (p.H, p.W):
            raise ValueError("batch images must be contiguous and match their plans")
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    fp = (ctypes.c_void_p * n)(*[f.data_ptr() for f in fs])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    nat.check(nat.lib().bf_execute_batch(n, hp, fp, op, _stream_ptr(stream)), "bf_execute_batch")
    return outs


def bf_get_info(plan: Plan) -> Info:
    i = nat.bf_info()
    nat.check(nat.lib().bf_get_info(plan.handle, ctypes.byref(i)), "bf_get_info")
    return Info(**{k: getattr(i, k) for k, _ in nat.bf_info._fields_})


def bf_get_sets(plan: Plan):
    """(T, N, M) numpy arrays, one entry per parameter set."""
    import numpy as np
    n = bf_get_info(plan).n_sets
    T = np.empty(n, np.float32)
    N = np.empty(n, np.int32)
    M = np.empty(n, np.int32)
    nat.check(nat.lib().bf_get_sets(plan.handle, T.ctypes.data, N.ctypes.data, M.ctypes.data, n),
              "bf_get_sets")
    return T, N, M


def bf_get_device_status(plan: Plan) -> int:
    bits = ctypes.c_uint()
    code = nat.lib().bf_get_device_status(plan.handle, ctypes.byref(bits))
    if code not in (nat.BF_OK, nat.BF_ERR_DEVICE_STATUS):
        nat.check(code, "bf_get_device_status")
    return bits.value


def bf_set_timing(plan: Plan, on: bool = True):
    nat.check(nat.lib().bf_set_timing(plan.handle, 1 if on else 0), "bf_set_timing")


def bf_get_timing(plan: Plan):
    """(ms_K1, ms_K2, ms_K3, ms_recheck) summed over the timed executes, and
    their count."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int()
    nat.check(nat.lib().bf_get_timing(plan.handle, ms, ctypes.byref(n)), "bf_get_timing")
    return (ms[0], ms[1], ms[2], ms[3]), n.value


def bf_destroy(plan: Plan):
    plan.close()


def bf_maxmin(f, R: int, stream=None):
    """Windowed max and min images (Prop. MAX-FILTER)."""
    import torch
    _check_image(f, "f")
    Mx = torch.empty_like(f)
    mn = torch.empty_like(f)
    if not (Mx.stride(0) == f.stride(0)):
        Mx = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
        mn = torch.empty_strided(f.shape, f.stride(), dtype=f.dtype, device=f.device)
    nat.check(nat.lib().bf_maxmin(f.data_ptr(), f.shape[0], f.shape[1], f.stride(0), int(R),
                                  Mx.data_ptr(), mn.data_ptr(), _stream_ptr(stream)), "bf_maxmin")
    return Mx, mn


def _autograd_fn():
    import torch

    class BilateralFilter(torch.autograd.Function):
        """out = bf_execute(f); backward = bf_backward (T, N, M held fixed)."""

        @staticmethod
        def forward(ctx, f, plan):
            out = bf_execute(plan, f.contiguous())
            ctx.plan = plan
            ctx.save_for_backward(f)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            (f,) = ctx.saved_tensors
            g = bf_backward(ctx.plan, f.contiguous(), grad_out.contiguous())
            return g, None

    return BilateralFilter


_BF = None


def bilateral_filter(f, plan: Plan):
    """Differentiable filter of a 2-D float32 CUDA tensor with a plan."""
    global _BF
    if _BF is None:
        _BF = _autograd_fn()
    return _BF.apply(f, plan)


def bf_test_stall(plan: Plan, on: bool = True):
    """Makes the plan's tensor-core forward run out a bounded wait (tests of
    the failure path; see include/bf.h)."""
    nat.check(nat.lib().bf_test_stall(plan.handle, 1 if on else 0), "bf_test_stall")
