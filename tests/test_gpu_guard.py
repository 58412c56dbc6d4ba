"""GPU check of the denominator guard (the paper is silent; where den <=
1e-6 of the clipped spatial mass the output is f(x)), on the images the
oracle's guard pins use: outliers in a zero field at the image border whose
den, by the plain-Python direct sum, is clearly negative (the guard fires)
or clearly positive (it does not).  The GPU's count of guarded outputs must
equal the oracle's, the guarded outputs must be f bit for bit, and the
others must match the oracle as usual.  FP32 planes run the fused FIR;
16-bit planes reach the guard through the FP32 recheck (every output whose
den is under 5 % of its mass is recomputed there, and the guard is decided
on that den)."""
import numpy as np
import pytest

import oracle
from test_oracle_guard import SS, SR, EPS, T, R, nm_py, outlier_height

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build
    build.build()
    import paper_1203_5128_gb300 as m
    return m


SPOTS = [(1, 1, -0.005), (0, 30, -0.003), (59, 78, 0.002), (30, 79, -0.002),
         (59, 40, 0.02), (1, 60, -0.005), (30, 20, 0.01)]


@pytest.mark.parametrize("planes", ["fp32", "fp16"])
def test_guard_count_and_fallback_on_gpu(bf, planes):
    import torch
    H, W = 60, 80
    N, M = nm_py()
    f = np.zeros((H, W))
    for i, j, ratio in SPOTS:
        f[i, j] = outlier_height(ratio, i, j, H, W, N, M)
    f32 = f.astype(np.float32)
    p = oracle.resolve(f32, SS, SR, EPS, t_mode="fixed", t_fixed=T, rule="trunc")
    assert (p.N[0, 0], p.M[0, 0]) == (N, M) and p.R == R
    ref, _, den, nfb = oracle.shiftable(f32, SS, SR, p, return_parts=True)
    assert 0 < nfb < len(SPOTS)
    plan = bf.bf_plan(H, W, SS, SR, EPS, t_mode="fixed", t_fixed=T, trunc_rule="trunc",
                      plane_dtype=planes)
    out = bf.bf_execute(plan, torch.from_numpy(f32).cuda())
    torch.cuda.synchronize()
    info = bf.bf_get_info(plan)
    o = out.cpu().numpy()
    guarded = [(i, j) for i, j, _ in SPOTS if ref[i, j] == f32[i, j] and den[i, j] <= 0]
    print("%s: GPU guarded %d, oracle %d" % (planes, info.n_guarded, nfb))
    assert info.n_guarded == nfb == len(guarded)
    for i, j in guarded:
        assert o[i, j] == f32[i, j]
    # the outliers the guard spares sit at den of 0.2 - 2 % of their mass, where
    # out = num / den is large: relative bar there (FP32 on both paths:
    # the 16-bit path rechecks them), the usual bar elsewhere
    mask = np.ones_like(o, dtype=bool)
    for i, j, _ in SPOTS:
        mask[i, j] = False
        if (i, j) not in guarded:
            assert abs(o[i, j] - ref[i, j]) <= 1e-3 * abs(ref[i, j])
    err = np.abs(o.astype(np.float64) - ref)[mask]
    assert err.max() <= (1e-3 if planes == "fp32" else 0.5)


def test_fp16_without_recheck_guards_negative_den(bf):
    """16-bit planes with the FP32 recheck off (lowp_recheck = 0): K3-tc's
    own guard takes the outputs whose den is negative -- here the two
    outliers at den = -0.5 % of their mass, below the FP16 rounding bound of
    den (4 u mass, u = 2^-11: 0.2 %) -- and outputs f there; nothing is
    listed for a recheck that the plan does not run."""
    import torch
    H, W = 60, 80
    N, M = nm_py()
    f = np.zeros((H, W))
    for i, j, ratio in SPOTS:
        f[i, j] = outlier_height(ratio, i, j, H, W, N, M)
    f32 = f.astype(np.float32)
    plan = bf.bf_plan(H, W, SS, SR, EPS, t_mode="fixed", t_fixed=T, trunc_rule="trunc",
                      plane_dtype="fp16", lowp_recheck=0.0)
    out = bf.bf_execute(plan, torch.from_numpy(f32).cuda())
    torch.cuda.synchronize()
    assert bf.bf_get_device_status(plan) == 0
    info = bf.bf_get_info(plan)
    o = out.cpu().numpy()
    assert np.all(np.isfinite(o))
    assert info.n_rechecked == 0
    clear = [(i, j) for i, j, ratio in SPOTS if ratio <= -0.005]
    assert info.n_guarded >= len(clear) >= 2
    for i, j in clear:
        assert o[i, j] == f32[i, j]
