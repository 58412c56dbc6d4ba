"""GPU parity of the O(1) non-local means with a small patch (Sec. 6, eqs.
(NL1), (NL2); bf_options.patch_mask) against the FP64 oracle's direct sums
with the same T, N, M, through the C ABI.

T (Algorithm 1), N and M come from the same K1 / K2 as the bilateral filter
and must be equal.  The FP32 planes carry the bilateral filter's FP32 bar:
1e-3 gray levels where den is a large part of the window's mass, plus FP32
roundoff times the pixel's condition number mass / den times T elsewhere
(the kernel weights of the multi-index terms sum to at most 1, as the
bilateral filter's do).
"""
import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

pytestmark = pytest.mark.gpu

CENTRE, RIGHT, DOWN, LEFT, UP = 1 << 4, 1 << 5, 1 << 7, 1 << 3, 1 << 1
P3 = CENTRE | RIGHT | DOWN
P5 = CENTRE | RIGHT | DOWN | LEFT | UP


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


def mass_at(g, R, ys, xs, H, W):
    def line(i, n):
        return g[max(0, i - R) - i + R: min(n - 1, i + R) - i + R + 1].sum()
    return np.array([line(y, H) * line(x, W) for y, x in zip(ys, xs)])


def run(bf, f, ss, sr, eps, mask, spatial, mode="global"):
    import torch
    H, W = f.shape
    kw = dict(t_mode=mode, trunc_rule="alg2", spatial=spatial)
    if mode == "fixed":
        kw["t_fixed"] = 255.0
    plan = bf.bf_plan(H, W, ss, sr, eps, patch_mask=mask, **kw)
    out = bf.bf_execute(plan, to_dev(f))
    torch.cuda.synchronize()
    assert bf.bf_get_device_status(plan) == 0
    sp = "box" if spatial == "box" else "fir"
    p = oracle.resolve(f, ss, sr, eps, t_mode=mode, rule="alg2", spatial=sp,
                       t_fixed=255.0 if mode == "fixed" else None)
    T, N, M = bf.bf_get_sets(plan)
    assert T[0] == p.T[0, 0] and N[0] == p.N[0, 0] and M[0] == p.M[0, 0]
    return plan, out.cpu().numpy().astype(np.float64), p, sp


def check(f, out, ss, sr, p, mask, sp, points=None, what=""):
    H, W = f.shape
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = points
    ref, _, den, _ = oracle.nlm_direct(f, ss, sr, p, mask, points=(ys, xs), spatial=sp,
                                       return_parts=True)
    g = oracle.spatial_taps(ss, p.R, sp)
    mass = mass_at(g, p.R, ys, xs, H, W)
    err = np.abs(out[ys, xs] - ref)
    tol = 1e-3 + 2.0 ** -22 * (mass / np.maximum(den, 1e-300)) * float(p.T.max())
    well = den > 0.05 * mass
    K = int(p.N[0, 0] - 2 * p.M[0, 0] + 1)
    print("nlm %s: N=%d M=%d K=%d, max-abs %.3g gray levels (%.3g where den > 5%% of the mass), "
          "largest share of the bar %.3g" % (what, p.N[0, 0], p.M[0, 0], K, err.max(),
                                             err[well].max() if well.any() else 0.0,
                                             float(np.max(err / tol))))
    assert np.all(err <= tol)
    if well.any():
        assert np.max(err[well]) <= 1e-3


CASES = [
    # H, W, sigma_s (box: radius), sigma_r, eps, mask, spatial, mode
    (96, 80, 3.0, 40.0, 0.05, P3, "box", "global"),
    (64, 72, 1.5, 50.0, 0.02, P5, "gauss", "global"),
    (100, 37, 5.0, 40.0, 0.05, CENTRE | RIGHT, "box", "fixed"),
    (1, 90, 2.0, 45.0, 0.05, P3, "box", "global"),
    (90, 1, 2.0, 45.0, 0.05, P3, "box", "global"),
    (130, 70, 2.0, 150.0, 0.01, 0x1FF, "box", "global"),     # the full 3 x 3 patch (N = 2)
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_s%g_r%g_m%x_%s_%s" % (
    c[0], c[1], c[2], c[3], c[5], c[6], c[7]))
def test_nlm_matches_oracle(bf, case):
    H, W, ss, sr, eps, mask, spatial, mode = case
    f = synth.g8(H, W, seed=H + 2 * W)
    plan, out, p, sp = run(bf, f, ss, sr, eps, mask, spatial, mode)
    check(f, out, ss, sr, p, mask, sp, what=str(case))


def test_one_pixel_patch_is_the_bilateral_filter(bf):
    """patch_mask = centre only: the non-local means kernel computes the
    bilateral filter; it agrees with the bilateral path to FP32 roundoff."""
    import torch
    f = synth.g8(128, 96, seed=4)
    _, a, p, _ = run(bf, f, 2.0, 30.0, 0.01, CENTRE, "gauss")
    plan = bf.bf_plan(128, 96, 2.0, 30.0, 0.01, t_mode="global", trunc_rule="alg2")
    b = bf.bf_execute(plan, to_dev(f))
    torch.cuda.synchronize()
    assert np.max(np.abs(a - b.cpu().numpy())) < 1e-3


def test_nlm_512_sampled(bf):
    """512^2 G8, box search window of radius 5, sigma_r = 40 per patch
    pixel, eps = 5e-2, the 3-pixel patch: sampled outputs."""
    f = synth.g8(512, 512, seed=11)
    plan, out, p, sp = run(bf, f, 5.0, 40.0, 0.05, P3, "box")
    rng = np.random.default_rng(3)
    ys = np.concatenate([rng.integers(0, 512, 200), [0, 511, 0, 511, 63, 64]])
    xs = np.concatenate([rng.integers(0, 512, 200), [0, 511, 511, 0, 32, 31]])
    check(f, out, 5.0, 40.0, p, P3, sp, points=(ys, xs), what="512^2 sampled")


def test_nlm_rejects_unsupported(bf):
    from paper_1203_5128_gb300 import _native as nat
    for kw, code in [(dict(patch_mask=RIGHT), nat.BF_ERR_INVALID_ARG),
                     (dict(patch_mask=P3, t_mode="tile"), nat.BF_ERR_NOT_SUPPORTED),
                     (dict(patch_mask=P3, plane_dtype="fp16"), nat.BF_ERR_NOT_SUPPORTED),
                     (dict(patch_mask=0x1FF, trunc_rule="trunc"), nat.BF_ERR_NOT_SUPPORTED)]:
        with pytest.raises(nat.BfError) as e:
            bf.bf_plan(64, 64, 2.0, 10.0, 0.0, **kw)
        assert e.value.code == code
