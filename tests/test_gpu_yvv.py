"""GPU parity of the recursive (Young-van Vliet) forward against the FP64
oracle's recursive mode.

The FP32 bar is the forward's: max-abs 1e-3 gray levels on 8-bit images.
Sizes are ragged, and cover both the 8- and 16-terms-per-pass kernel widths,
several passes, single rows and columns, and both FIXED and GLOBAL T.  At the full
4096 x 4096 size the oracle runs on crops: the recursion's response falls
below 3e-14 of its peak within 200 pixels at sigma_s = 8, so the outputs
200 pixels or more inside a crop's interior edges equal those of the whole
image (the crop keeps the image's own borders, where it touches them, and
the whole image's T, N and M).
"""
import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-3


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build
    build.build()
    import paper_1203_5128_gb300 as m
    return m


def run(bf, f, sigma_s, sigma_r, eps, **opts):
    import torch
    H, W = f.shape
    p = bf.bf_plan(H, W, sigma_s, sigma_r, eps, filter="yvv", **opts)
    out = bf.bf_execute(p, torch.from_numpy(np.ascontiguousarray(f, np.float32)).cuda())
    torch.cuda.synchronize()
    info = bf.bf_get_info(p)
    res = out.cpu().numpy().astype(np.float64)
    p.close()
    return res, info


# (H, W, sigma_s, sigma_r, eps, t_mode, rule): sigma_r 60 -> 8 terms per
# pass, 40 -> 16, 15 -> 16 x 4 passes, 10 -> 16 x 9 passes (caps on N)
CASES = [
    (37, 53, 0.8, 60.0, 0.01, "global", "alg2"),
    (96, 80, 2.0, 40.0, 0.0, "global", "trunc"),
    (130, 257, 5.0, 15.0, 0.01, "global", "alg2"),
    (71, 129, 3.0, 10.0, 0.01, "global", "chernoff"),
    (64, 96, 1.5, 30.0, 0.0, "fixed", "alg2"),
    (1, 77, 2.0, 30.0, 0.01, "global", "alg2"),
    (83, 1, 2.0, 30.0, 0.01, "global", "alg2"),
]


@pytest.mark.parametrize("H,W,ss,sr,eps,mode,rule", CASES)
def test_matches_oracle(bf, H, W, ss, sr, eps, mode, rule):
    f = synth.g8(H, W, seed=H * 1000 + W)
    kw = dict(t_mode=mode, trunc_rule=rule)
    okw = dict(t_mode=mode, rule=rule)
    if mode == "fixed":
        kw["t_fixed"] = 255.0
        okw["t_fixed"] = 255.0
    got, info = run(bf, f, ss, sr, eps, **kw)
    p = oracle.resolve(f, ss, sr, eps, **okw)
    assert (info.N, info.M) == (int(p.N[0, 0]), int(p.M[0, 0]))
    ref = oracle.shiftable(f, ss, sr, p, spatial="yvv")
    assert np.max(np.abs(got - ref)) <= TOL


def test_constant_image(bf):
    f = np.full((50, 70), 123.0, np.float32)
    got, info = run(bf, f, 3.0, 20.0, 0.01)
    assert info.N == 1
    assert np.max(np.abs(got - 123.0)) <= 1e-4


def test_deterministic(bf):
    import torch
    f = torch.from_numpy(synth.g8(200, 300, seed=4)).cuda()
    p = bf.bf_plan(200, 300, 4.0, 15.0, 0.01, filter="yvv")
    a = bf.bf_execute(p, f).cpu().numpy()
    b = bf.bf_execute(p, f).cpu().numpy()
    assert np.array_equal(a, b)
    p.close()


def test_rejections(bf):
    import torch
    with pytest.raises(bf.BfError):
        bf.bf_plan(64, 64, 2.0, 20.0, 0.01, filter="yvv", t_mode="tile")
    with pytest.raises(bf.BfError):
        bf.bf_plan(64, 64, 2.0, 20.0, 0.01, filter="yvv", plane_dtype="fp16")
    with pytest.raises(bf.BfError):
        bf.bf_plan(64, 64, 0.4, 20.0, 0.01, filter="yvv")
    p = bf.bf_plan(64, 64, 2.0, 20.0, 0.01, filter="yvv")
    f = torch.from_numpy(synth.g8(64, 64, seed=1)).cuda()
    bf.bf_execute(p, f)
    with pytest.raises(bf.BfError):
        bf.bf_backward(p, f, torch.ones_like(f))
    with pytest.raises(bf.BfError):
        bf.bf_execute_batch([p], [f])
    p.close()


def test_full_size_crops(bf):
    """4096 x 4096, sigma_s = 8, sigma_r = 10, Algorithm 2 with eps = 1e-2
    and exact T: a corner crop (keeps two image borders) and a central one."""
    H = W = 4096
    ss, sr, eps = 8.0, 10.0, 0.01
    f = synth.g8(H, W, seed=5)
    got, info = run(bf, f, ss, sr, eps)
    p = oracle.resolve(f, ss, sr, eps, t_mode="global", rule="alg2")
    assert (info.N, info.M) == (int(p.N[0, 0]), int(p.M[0, 0]))
    c, keep = 640, 200
    # corner: rows/cols [0, c); exact where >= keep from the inner edges
    ref = oracle.shiftable(f[:c, :c], ss, sr, p, spatial="yvv")
    e1 = np.max(np.abs(got[:c - keep, :c - keep] - ref[:c - keep, :c - keep]))
    # centre
    y0 = x0 = (H - c) // 2
    ref = oracle.shiftable(f[y0:y0 + c, x0:x0 + c], ss, sr, p, spatial="yvv")
    e2 = np.max(np.abs(got[y0 + keep:y0 + c - keep, x0 + keep:x0 + c - keep]
                       - ref[keep:c - keep, keep:c - keep]))
    assert max(e1, e2) <= TOL
