"""The bounded-wait path of the tensor-core forward, run on the GPU without a
fault: bf_test_stall makes the kernel's MMA-issuing thread wait for a
barrier nothing arrives on.  The wait runs out after spin_limit polls, the
CTA stops its roles (no MMA has been issued, so nothing is left to drain),
frees its tensor memory and returns; the device status word reports
BF_DEV_TIMEOUT, and the context stays usable: the next execute of the same
plan, with the stall off, gives the usual result."""
import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build
    build.build()
    import paper_1203_5128_gb300 as m
    return m


@pytest.mark.parametrize("planes", ["fp16", "bf16"])
def test_bounded_wait_times_out_and_recovers(bf, planes):
    import torch
    from paper_1203_5128_gb300 import _native as nat
    H, W = 128, 64                                 # two tiles: two CTAs stall
    f_np = synth.g8(H, W, seed=12)
    f = torch.from_numpy(f_np).cuda()
    plan = bf.bf_plan(H, W, 2.0, 20.0, 0.01, plane_dtype=planes, spin_limit=1 << 16)
    bf.bf_test_stall(plan, True)
    bf.bf_execute(plan, f)
    torch.cuda.synchronize()
    bits = bf.bf_get_device_status(plan)           # reads and clears the word
    assert bits & nat.BF_DEV_TIMEOUT
    bf.bf_test_stall(plan, False)
    out = bf.bf_execute(plan, f)
    torch.cuda.synchronize()
    assert bf.bf_get_device_status(plan) == 0
    p = oracle.resolve(f_np, 2.0, 20.0, 0.01, t_mode="global")
    err = np.max(np.abs(out.cpu().numpy() - oracle.shiftable(f_np, 2.0, 20.0, p)))
    assert err <= {"fp16": 0.5, "bf16": 2.0}[planes]


def test_stall_needs_the_tensor_core_path(bf):
    from paper_1203_5128_gb300 import _native as nat
    plan = bf.bf_plan(64, 64, 2.0, 20.0, 0.01)     # FP32 planes
    with pytest.raises(nat.BfError) as e:
        bf.bf_test_stall(plan, True)
    assert e.value.code == nat.BF_ERR_NOT_SUPPORTED
