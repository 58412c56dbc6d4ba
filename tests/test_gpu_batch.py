"""GPU tests of bf_execute_batch (K1 batched, K2 batched, persistent K4 fed
by a tile queue, captured in a CUDA graph).

The batch must reproduce n separate bf_execute calls bit for bit (the
forward's arithmetic does not depend on which tile shape serves an image),
on the first call and on later calls that reuse the captured graph with new
image contents; one image is also checked against the FP64 oracle.
"""
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


def make_batch(bf, specs, seed0, eps=0.01, modes=None):
    import torch
    plans, fs, nps = [], [], []
    for k, (H, W, ss, sr) in enumerate(specs):
        mode = modes[k % len(modes)] if modes else "global"
        kw = dict(t_mode=mode)
        if mode == "fixed":
            kw["t_fixed"] = 255.0
        plans.append(bf.bf_plan(H, W, ss, sr, eps, **kw))
        a = synth.g8(H, W, seed=seed0 + k)
        nps.append(a)
        fs.append(torch.from_numpy(a).cuda())
    return plans, fs, nps


def separate(bf, plans, fs):
    import torch
    outs = [bf.bf_execute(p, f) for p, f in zip(plans, fs)]
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def test_batch_matches_separate_calls_bitwise(bf):
    import torch
    rng = np.random.default_rng(11)
    specs = [(int(rng.integers(40, 300)), int(rng.integers(40, 300)),
              float(rng.uniform(1.0, 12.0)), float(rng.uniform(10.0, 60.0))) for _ in range(8)]
    plans, fs, nps = make_batch(bf, specs, 200, modes=["global", "tile", "fixed"])
    ref = separate(bf, plans, fs)
    outs = bf.bf_execute_batch(plans, fs)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert np.array_equal(o.cpu().numpy(), r)
    # graph reuse with new contents in the same buffers
    for k, f in enumerate(fs):
        f.copy_(torch.from_numpy(synth.g8(*f.shape, seed=900 + k)).cuda())
    bf.bf_execute_batch(plans, fs, outs)
    torch.cuda.synchronize()
    ref2 = separate(bf, plans, fs)
    for o, r in zip(outs, ref2):
        assert np.array_equal(o.cpu().numpy(), r)
    # one image against the oracle
    H, W, ss, sr = specs[0]
    f0 = fs[0].cpu().numpy()
    p = oracle.resolve(f0, ss, sr, 0.01, t_mode="global")
    ref0 = oracle.shiftable(f0, ss, sr, p)
    assert np.max(np.abs(outs[0].cpu().numpy() - ref0)) <= 1e-3
    for p_ in plans:
        p_.close()


def test_batch_workload_bitwise(bf):
    """64 G8 images, sides uniform in [128, 2048], sigma_s in [2, 16],
    sigma_r in [10, 60], eps = 1e-2, exact T: one graph launch vs 64
    bf_execute calls."""
    import torch
    specs = synth.batch_specs(64, seed=3)
    plans, fs, _ = make_batch(bf, specs, 3000)
    ref = separate(bf, plans, fs)
    outs = bf.bf_execute_batch(plans, fs)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert np.array_equal(o.cpu().numpy(), r), k
    for p_ in plans:
        p_.close()


def test_batch_rejects_reduced_precision(bf):
    import torch
    p = bf.bf_plan(64, 64, 2.0, 20.0, 0.01, plane_dtype="fp16")
    f = torch.zeros((64, 64), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_execute_batch([p], [f])


def test_batch_rejects_a_plan_named_twice(bf):
    import torch
    p = bf.bf_plan(64, 64, 2.0, 20.0, 0.01)
    f = torch.zeros((64, 64), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_execute_batch([p, p], [f, f.clone()])
    p.close()
