"""The precision workload at its stated size: one 4096 x 4096 G16 image
(16-bit range), sigma_s = 8 (R = 24), sigma_r = 2000, exact T of the whole
image (Algorithm 1), no truncation (eps = 0, so K = N + 1 terms: the large-N
end of Sec. 1.3, N = ceil(4 T^2 / (pi^2 sigma_r^2)) up to 436 at T = 65535),
filtered with FP32, BF16 and FP16 planes.

Every output of rows 0..1023 is compared with the FP64 oracle run on rows
0..1047 of the image (each output depends on the rows within R of it) with
the whole image's T, N, M.  Errors are in 16-bit gray levels.  The bars are
the 8-bit workloads' bars at the same fraction of the range (x 257): FP32
1e-3 x 257, FP16 0.5 x 257, BF16 2 x 257.  An FP16 significand holds 11
bits, so its rounding alone is several 16-bit gray levels; the measured
error of each variant is printed.
"""
import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu

H = W = 4096
SS, SR, EPS, VR, SEED = 8.0, 2000.0, 0.0, 65535.0, 2
ROWS = 1024
BARS = {"fp32": 1e-3 * 257, "fp16": 0.5 * 257, "bf16": 2.0 * 257}


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build
    build.build()
    import paper_1203_5128_gb300 as m
    return m


@pytest.fixture(scope="module")
def reference():
    f = synth.g16(H, W, seed=SEED)
    p = oracle.resolve(f, SS, SR, EPS, t_mode="global", rule="alg2", value_range=VR)
    R = p.R
    crop = np.ascontiguousarray(f[:ROWS + R])
    ref, _, den, _ = oracle.shiftable(crop, SS, SR, p, return_parts=True)
    return f, p, ref[:ROWS], den[:ROWS]


@pytest.mark.parametrize("planes", ["fp32", "bf16", "fp16"])
def test_precision_workload_rows(bf, reference, planes):
    import torch
    f, p, ref, den = reference
    plan = bf.bf_plan(H, W, SS, SR, EPS, t_mode="global", trunc_rule="alg2", value_range=VR,
                      plane_dtype=planes)
    out = bf.bf_execute(plan, torch.from_numpy(f).cuda())
    torch.cuda.synchronize()
    assert bf.bf_get_device_status(plan) == 0
    T, N, M = bf.bf_get_sets(plan)
    assert T[0] == p.T[0, 0] and N[0] == p.N[0, 0] and M[0] == p.M[0, 0]
    info = bf.bf_get_info(plan)
    err = np.abs(out[:ROWS].cpu().numpy().astype(np.float64) - ref)
    print("precision 4096^2 G16 %s (T=%g N=%d K=%d): max-abs %.4g, mean %.3g 16-bit gray "
          "levels over %d outputs (%d rechecked in FP32)" % (
              planes, T[0], N[0], info.K, err.max(), err.mean(), err.size, info.n_rechecked))
    assert np.max(err) <= BARS[planes]
