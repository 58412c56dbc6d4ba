"""GPU parity of the hand-written adjoint (K5) through bf_backward.

Checks: the gradient of L = sum(u * out) against the FP64 oracle gradient
(shiftable form, which the oracle pins tie to its direct-form derivative and
to central differences) with the same T, N, M, within 1e-3 of max |grad|;
central finite differences of the GPU forward itself along a random
direction (T fixed, so N and M cannot move); the torch.autograd.Function;
and the differentiation workload (batch of 512 x 512 G8 images, sigma_s = 4,
sigma_r = 25, eps = 1e-2, w ~ N(0, 1)).
"""
import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-3


@pytest.fixture(scope="module")
def bf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1203_5128_gb300 import build
    build.build()
    import paper_1203_5128_gb300 as m
    return m


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_grad(bf, f, u, ss, sr, eps, **kw):
    import torch
    H, W = f.shape
    plan = bf.bf_plan(H, W, ss, sr, eps, **kw)
    fd = to_dev(f)
    bf.bf_execute(plan, fd)
    g = bf.bf_backward(plan, fd, to_dev(u))
    torch.cuda.synchronize()
    return plan, g.cpu().numpy().astype(np.float64)


CASES = [
    # H, W, sigma_s, sigma_r, eps, mode, tile
    (40, 56, 1.5, 25.0, 0.01, "global", 64),
    (70, 45, 2.0, 15.0, 0.01, "fixed", 64),
    (128, 96, 1.2, 30.0, 0.01, "tile", 64),
    (33, 65, 4.0, 25.0, 0.01, "global", 64),     # R = 12, ragged
    (50, 50, 8.0, 40.0, 0.05, "global", 64),     # R = 24 (scalar form)
    (96, 130, 5.0, 30.0, 0.01, "global", 64),    # R = 15: 5 input steps
    (80, 70, 6.0, 40.0, 0.01, "tile", 64),       # R = 18: 6 steps, per-tile T
    (200, 150, 4.0, 20.0, 0.01, "tile", 64),     # R = 12, several T-tiles per halo
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_s%g_r%g_%s" % (c[0], c[1], c[2], c[3], c[5]))
def test_backward_matches_oracle(bf, case):
    H, W, ss, sr, eps, mode, tile = case
    f = synth.g8(H, W, seed=H + W)
    u = np.random.default_rng(H * W).normal(size=(H, W))
    kw = dict(t_mode=mode, t_tile=tile)
    if mode == "fixed":
        kw["t_fixed"] = 255.0
    plan, g = gpu_grad(bf, f, u.astype(np.float32), ss, sr, eps, **kw)
    p = oracle.resolve(f, ss, sr, eps, t_mode=mode, t_tile=tile,
                       t_fixed=255.0 if mode == "fixed" else None)
    T, N, M = bf.bf_get_sets(plan)
    assert np.array_equal(N, p.N.ravel().astype(np.int32)) and np.array_equal(M, p.M.ravel().astype(np.int32))
    ref = oracle.grad_shiftable(f, u.astype(np.float32).astype(np.float64), ss, sr, p)
    err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    print("%s: max |grad - oracle| / max |oracle| = %.2e" % (case, err))
    assert err <= REL


def test_backward_finite_differences(bf):
    """<grad L, v> against (L(f + h v) - L(f - h v)) / 2h of the GPU forward
    (T fixed at 255 so that N and M are constant; sums in FP64)."""
    import torch
    H, W, ss, sr, eps = 96, 80, 2.0, 20.0, 0.01
    f = synth.g8(H, W, seed=31).astype(np.float64)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(H, W))
    v = rng.normal(size=(H, W))
    plan, g = gpu_grad(bf, f, u.astype(np.float32), ss, sr, eps, t_mode="fixed", t_fixed=255.0)
    h = 0.05

    def L(x):
        out = bf.bf_execute(plan, to_dev(x))
        torch.cuda.synchronize()
        return float(np.sum(u.astype(np.float32).astype(np.float64) * out.cpu().numpy()))
    fd = (L(f + h * v) - L(f - h * v)) / (2 * h)
    an = float(np.sum(g * v))
    print("directional: analytic %.6f  fd %.6f" % (an, fd))
    assert abs(an - fd) <= 2e-3 * abs(an) + 1e-2


def test_autograd_function(bf):
    import torch
    H, W = 64, 72
    f = to_dev(synth.g8(H, W, seed=3)).requires_grad_(True)
    w = to_dev(np.random.default_rng(0).normal(size=(H, W)))
    plan = bf.bf_plan(H, W, 2.0, 25.0, 0.01)
    loss = (bf.bilateral_filter(f, plan) * w).sum()
    (gf,) = torch.autograd.grad(loss, f)
    direct = bf.bf_backward(plan, f.detach(), w)
    torch.cuda.synchronize()
    assert torch.equal(gf, direct)


def test_backward_before_forward_is_an_error(bf):
    import torch
    plan = bf.bf_plan(16, 16, 1.0, 20.0, 0.0)
    x = torch.zeros((16, 16), device="cuda")
    with pytest.raises(bf.BfError):
        bf.bf_backward(plan, x, x)


def test_differentiation_workload(bf):
    """Batch of 512^2 G8 images, sigma_s = 4, sigma_r = 25, eps = 1e-2,
    global T; two images of the batch checked against the FP64 oracle."""
    import torch
    H = W = 512
    ss, sr, eps = 4.0, 25.0, 0.01
    wgt = synth.weights_normal((H, W), seed=4)
    for b in (0, 7):
        f = synth.g8(H, W, seed=100 + b)
        plan, g = gpu_grad(bf, f, wgt, ss, sr, eps, t_mode="global")
        p = oracle.resolve(f, ss, sr, eps, t_mode="global")
        ref = oracle.grad_shiftable(f, wgt.astype(np.float64), ss, sr, p)
        err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
        print("image %d: N=%d M=%d rel err %.2e" % (b, p.N[0, 0], p.M[0, 0], err))
        assert err <= REL
