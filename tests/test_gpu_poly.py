"""GPU parity of the raised-polynomial range kernel (eq. (RPconv), Sec. 1.3)
against the FP64 oracle's direct sum of eq. (BF) with the same kernel, T
and N, through the C ABI.

T (the range of f over each parameter set's region) and N are exact integer
decisions taken in FP64 on both sides from the same float values, so they
must be equal.  The outputs carry FP32 roundoff of the basis expansion: the
bar is 1e-3 gray levels plus FP32 roundoff (2^-24) times n (the 2N + 1 terms)
times the pixel's condition number mass / den times T, the same form as the
FP32 cosine path's bar at large windows; it is 1e-3 wherever den is a large
part of the window's mass.
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


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def mass_at(g, R, ys, xs, H, W):
    def line(i, n):
        return g[max(0, i - R) - i + R: min(n - 1, i + R) - i + R + 1].sum()
    return np.array([line(y, H) * line(x, W) for y, x in zip(ys, xs)])


def run(bf, f, ss, sr, mode, tile=64, spatial="gauss", vr=255.0, tf=None, **kw):
    import torch
    H, W = f.shape
    opts = dict(t_mode=mode, t_tile=tile, range_kernel="poly", spatial=spatial, value_range=vr)
    if tf is not None:
        opts["t_fixed"] = tf
    opts.update(kw)
    plan = bf.bf_plan(H, W, ss, sr, 0.0, **opts)
    out = bf.bf_execute(plan, to_dev(f))
    torch.cuda.synchronize()
    sp = "box" if spatial == "box" else "fir"
    p = oracle.resolve(f, ss, sr, t_mode=mode, t_tile=tile, value_range=vr, t_fixed=tf,
                       kernel="poly", spatial=sp)
    return plan, out.cpu().numpy().astype(np.float64), p, sp


def check(bf, plan, out, f, ss, sr, p, sp, points=None, what=""):
    T, N, M = bf.bf_get_sets(plan)
    assert np.array_equal(T, p.T.ravel()), (T, p.T)
    assert np.array_equal(N, p.N.ravel().astype(np.int32)), (N, p.N)
    assert np.all(M == 0)
    H, W = f.shape
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = points
    ref, _, den, nfb = oracle.poly_direct(f, ss, sr, p, points=(ys, xs), return_parts=True,
                                          spatial=sp)
    g = oracle.spatial_taps(ss, p.R, sp)
    mass = mass_at(g, p.R, ys, xs, H, W)
    err = np.abs(out[ys, xs] - ref)
    nmax = 2 * int(p.N.max()) + 1
    tol = 1e-3 + 2.0 ** -24 * nmax * (mass / np.maximum(den, 1e-300)) * float(p.T.max())
    well = den > 0.05 * mass
    print("poly %s: max-abs %.3g gray levels (%.3g where den > 5%% of the mass), N up to %d, "
          "largest share of the bar %.3g" % (what, err.max(), err[well].max() if well.any() else 0,
                                             int(p.N.max()), float(np.max(err / tol))))
    assert np.all(err <= tol)
    if well.any():
        assert np.max(err[well]) <= 1e-3
    return err


CASES = [
    # H, W, sigma_s, sigma_r, mode, tile, spatial
    (256, 200, 3.0, 30.0, "fixed", 64, "gauss"),
    (200, 150, 2.0, 40.0, "global", 64, "gauss"),
    (256, 320, 4.0, 25.0, "tile", 64, "gauss"),
    (130, 33, 8.0, 30.0, "global", 64, "gauss"),         # R = 24, ragged tiles
    (120, 90, 5.0, 30.0, "tile", 64, "box"),             # box spatial filter (Sec. 4)
    (1, 90, 2.0, 35.0, "global", 64, "gauss"),
    (90, 1, 2.0, 35.0, "global", 64, "gauss"),
    (64, 64, 12.0, 50.0, "tile", 64, "gauss"),           # R = 36
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_s%g_r%g_%s_%s" % (c[0], c[1], c[2],
                                                                               c[3], c[4], c[6]))
def test_poly_matches_oracle(bf, case):
    H, W, ss, sr, mode, tile, spatial = case
    f = synth.g8(H, W, seed=H * 3 + W)
    tf = 255.0 if mode == "fixed" else None
    plan, out, p, sp = run(bf, f, ss, sr, mode, tile, spatial, tf=tf)
    assert bf.bf_get_device_status(plan) == 0
    check(bf, plan, out, f, ss, sr, p, sp, what=str(case))


def test_poly_16bit_image(bf):
    """16-bit range (G16): the values are mapped onto [-1, 1] per set, so
    the arithmetic is that of the 8-bit case (bar x 257)."""
    f = synth.g16(96, 80, seed=2)
    plan, out, p, sp = run(bf, f, 2.0, 6000.0, "global", vr=65535.0)
    T, N, _ = bf.bf_get_sets(plan)
    assert np.array_equal(T, p.T.ravel()) and np.array_equal(N, p.N.ravel().astype(np.int32))
    ref = oracle.poly_direct(f, 2.0, 6000.0, p)
    err = np.abs(out - ref)
    print("poly 16-bit: max-abs %.3g (16-bit gray levels), N=%d" % (err.max(), N[0]))
    assert err.max() <= 257 * 1e-3


def test_poly_constant_and_flat_tiles(bf):
    """A flat T-tile has T = 0, N = 1 and passes its values through."""
    g = np.full((128, 192), 77.0, np.float32)
    g[:, 150:] = 140.0
    plan, out, p, sp = run(bf, g, 2.0, 30.0, "tile", 64)
    T, N, _ = bf.bf_get_sets(plan)
    assert T[0] == 0.0 and N[0] == 1
    assert np.max(np.abs(out[:64, :64] - 77.0)) < 1e-4
    check(bf, plan, out, g, 2.0, 30.0, p, sp, what="flat tiles")


def test_poly_order_cap_passes_through(bf):
    from paper_1203_5128_gb300 import _native as nat
    f = synth.g8(128, 128, seed=3)
    plan, out, p, sp = run(bf, f, 2.0, 10.0, "global", n_max=40)
    assert np.array_equal(out, f.astype(np.float64))
    assert bf.bf_get_device_status(plan) & nat.BF_DEV_ORDER_TOO_LARGE


def test_poly_1024_sampled(bf):
    """1024^2 G8, sigma_s = 3, sigma_r = 30, range T per 64 x 64 T-tile,
    sampled outputs (random, corners, T-tile seams)."""
    f = synth.g8(1024, 1024, seed=1)
    plan, out, p, sp = run(bf, f, 3.0, 30.0, "tile", 64)
    rng = np.random.default_rng(5)
    ys = np.concatenate([rng.integers(0, 1024, 300), [0, 1023, 0, 1023, 63, 64, 512]])
    xs = np.concatenate([rng.integers(0, 1024, 300), [0, 1023, 1023, 0, 64, 63, 512]])
    check(bf, plan, out, f, 3.0, 30.0, p, sp, points=(ys, xs), what="1024^2 sampled")


def test_poly_rejects_unsupported(bf):
    from paper_1203_5128_gb300 import _native as nat
    for kw in [dict(plane_dtype="fp16"), dict(filter="yvv"), dict(t_mode="fixed", t_fixed=100.0)]:
        with pytest.raises(nat.BfError) as e:
            bf.bf_plan(64, 64, 2.0, 30.0, 0.0, range_kernel="poly", **kw)
        assert e.value.code == nat.BF_ERR_NOT_SUPPORTED
