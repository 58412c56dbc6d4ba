"""GPU tests of bf_execute_batch (K1 batched, K2 batched, persistent K4 fed
by a tile queue, captured in a CUDA graph).

The batch must reproduce n separate bf_execute calls bit for bit (the
forward's arithmetic does not depend on which tile shape serves an image),
on the first call and on later calls that reuse the captured graph with new
image contents, with FP32 and 16-bit planes; images are also checked against
the FP64 oracle (one of the mixed batch, every image of the 64-image
workload at sampled pixels).
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


def test_batch_reduced_precision_bitwise(bf):
    """16-bit plans (FP16 and BF16 planes on the tensor cores, exact T of the
    image or per 128 x 128 T-tile) in one batch with FP32 plans: each image
    equals its own bf_execute bit for bit (the recheck lists depend on the
    launch order, its per-pixel results do not), on the first call and on a
    replay of the graph with new contents."""
    import torch
    rng = np.random.default_rng(17)
    plans, fs = [], []
    kinds = [("fp16", "global"), ("bf16", "tile"), ("fp32", "global"), ("fp16", "tile"),
             ("bf16", "global"), ("fp32", "tile")]
    for k, (planes, mode) in enumerate(kinds):
        H, W = int(rng.integers(130, 400)), int(rng.integers(100, 380))
        ss, sr = float(rng.uniform(1.5, 8.0)), float(rng.uniform(10.0, 40.0))
        kw = dict(t_mode=mode, plane_dtype=planes)
        if mode == "tile":
            kw["t_tile"] = 128
        plans.append(bf.bf_plan(H, W, ss, sr, 0.01, **kw))
        fs.append(torch.from_numpy(synth.g8(H, W, seed=500 + k)).cuda())
    for rep in range(2):
        if rep:
            for k, f in enumerate(fs):
                f.copy_(torch.from_numpy(synth.g8(*f.shape, seed=700 + k)).cuda())
        outs = bf.bf_execute_batch(plans, fs, None if rep == 0 else outs)
        torch.cuda.synchronize()
        ref = separate(bf, plans, fs)
        for k, (o, r) in enumerate(zip(outs, ref)):
            assert np.array_equal(o.cpu().numpy(), r), (rep, k, kinds[k])
    for p_ in plans:
        assert bf.bf_get_device_status(p_) == 0
        p_.close()


def test_batch_workload_fp16_every_image_vs_oracle(bf):
    """The 64-image workload with FP16 planes wherever the tensor-core kernel
    takes the radius (R <= 24) and FP32 planes elsewhere: bitwise equal to
    64 bf_execute calls, and every image against the FP64 oracle's direct
    form at sampled pixels (random, corners, borders): FP16 images within
    0.5 gray level, FP32 images (R > 24, with the FP32 recheck,
    fp32_recheck = 0.05) within 1e-3."""
    import torch
    specs = synth.batch_specs(64, seed=3)
    plans, fs, nps, kinds = [], [], [], []
    for k, (H, W, ss, sr) in enumerate(specs):
        planes = "fp16" if int(np.ceil(3 * ss)) <= 24 else "fp32"
        plans.append(bf.bf_plan(H, W, ss, sr, 0.01, plane_dtype=planes, fp32_recheck=0.05))
        a = synth.g8(H, W, seed=3000 + k)
        nps.append(a)
        fs.append(torch.from_numpy(a).cuda())
        kinds.append(planes)
    assert "fp16" in kinds and "fp32" in kinds
    ref = separate(bf, plans, fs)
    outs = bf.bf_execute_batch(plans, fs)
    torch.cuda.synchronize()
    worst = {"fp16": 0.0, "fp32": 0.0}
    for k, ((H, W, ss, sr), o, r) in enumerate(zip(specs, outs, ref)):
        o = o.cpu().numpy()
        assert np.array_equal(o, r), k
        p = oracle.resolve(nps[k], ss, sr, 0.01, t_mode="global")
        rng = np.random.default_rng(k)
        ys = np.concatenate([rng.integers(0, H, 24), [0, H - 1, 0, H - 1, H // 2]])
        xs = np.concatenate([rng.integers(0, W, 24), [0, W - 1, W - 1, 0, 0]])
        d = oracle.direct(nps[k], ss, sr, p, points=(ys, xs))
        err = float(np.max(np.abs(o[ys, xs] - d)))
        worst[kinds[k]] = max(worst[kinds[k]], err)
        assert err <= (0.5 if kinds[k] == "fp16" else 1e-3), (k, kinds[k], err)
    print("64-image batch vs the oracle at sampled pixels: max-abs FP16 %.3g, FP32 %.3g" % (
        worst["fp16"], worst["fp32"]))
    for p_ in plans:
        p_.close()


def test_batch_rejects_a_plan_named_twice(bf):
    import torch
    p = bf.bf_plan(64, 64, 2.0, 20.0, 0.01)
    f = torch.zeros((64, 64), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_execute_batch([p, p], [f, f.clone()])
    p.close()


def test_batch_fp32_recheck_large_windows(bf):
    """FP32 images with R > 24 in a batch: per-tile T (the persistent queue,
    then the FP32 recheck after it), image-wide T (the two-pass FIR on a
    launch of its own, then its recheck) and fixed T.  Bitwise equal to
    separate bf_execute calls, outputs listed for the recheck, and every
    output within 1e-3 of the FP64 oracle with the same T, N, M."""
    import torch
    specs = [(200, 180, 10.0, 8.0, "tile"), (150, 210, 9.0, 8.0, "global"),
             (120, 160, 11.0, 10.0, "fixed")]
    plans, fs, nps = [], [], []
    for k, (H, W, ss, sr, mode) in enumerate(specs):
        kw = dict(t_mode=mode, t_tile=64)
        if mode == "fixed":
            kw["t_fixed"] = 255.0
        plans.append(bf.bf_plan(H, W, ss, sr, 0.01, **kw))
        a = synth.g8(H, W, seed=4100 + k)
        nps.append(a)
        fs.append(torch.from_numpy(a).cuda())
    ref = separate(bf, plans, fs)
    listed = [bf.bf_get_info(p_).n_rechecked for p_ in plans]
    outs = bf.bf_execute_batch(plans, fs)
    torch.cuda.synchronize()
    assert sum(listed) > 0, listed
    for k, ((H, W, ss, sr, mode), o, r) in enumerate(zip(specs, outs, ref)):
        o = o.cpu().numpy()
        assert np.array_equal(o, r), k
        p = oracle.resolve(nps[k], ss, sr, 0.01, t_mode=mode, t_tile=64,
                           t_fixed=255.0 if mode == "fixed" else None)
        err = np.max(np.abs(o - oracle.shiftable(nps[k], ss, sr, p)))
        print("batch FP32 R=%d %s: %d outputs rechecked, max-abs %.3g" % (
            int(np.ceil(3 * ss)), mode, listed[k], err))
        assert err <= 1e-3, (k, err)
    for p_ in plans:
        p_.close()
