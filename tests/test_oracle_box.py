"""Pins of the oracle's box mode: the constant spatial filter of radius
sigma_s with the Gaussian range kernel, the setting in which Sec. 4 compares
SHIFTABLE-BF with BF2 (integral histograms work only for box filters; the
shiftable algorithm takes any spatial filter).

None of these tests calls the oracle's spatial filter to check itself:
sigma_r -> infinity is checked against running sums of an integral image,
the phi_eps filter and the Gaussian-range filter against pure-Python brute
force on tiny images, and the shiftable form against the direct form.
"""
from math import comb, sqrt

import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth


def small_image(H, W, seed):
    return synth.g8(H, W, seed).astype(np.float64)


def box_mean_integral(f, R):
    """Mean of f over the (2R+1)^2 square clipped to the image, from an
    integral image (four lookups per pixel: the O(1) running sums of a box
    filter)."""
    H, W = f.shape
    S = np.zeros((H + 1, W + 1))
    S[1:, 1:] = np.cumsum(np.cumsum(f, axis=0), axis=1)
    y0 = np.clip(np.arange(H) - R, 0, H)[:, None]
    y1 = np.clip(np.arange(H) + R + 1, 0, H)[:, None]
    x0 = np.clip(np.arange(W) - R, 0, W)[None, :]
    x1 = np.clip(np.arange(W) + R + 1, 0, W)[None, :]
    total = S[y1, x1] - S[y0, x1] - S[y1, x0] + S[y0, x0]
    count = (y1 - y0) * (x1 - x0)
    return total / count


def phi_brute(s, N, M, sigma_r):
    """phi_eps(s) = sum_{n=M}^{N-M} 2^-N C(N, n) cos((2n - N) s / (sqrt(N) sigma_r))
    (eqs. (expansion), (approx)), with exact integer binomials."""
    acc = 0.0
    for n in range(M, N - M + 1):
        acc += comb(N, n) / 2.0 ** N * np.cos((2 * n - N) * s / (sqrt(N) * sigma_r))
    return acc


def test_radius_is_sigma_s():
    """Sec. 4 names the radius of the box sigma_s: R = sigma_s, an integer."""
    f = small_image(20, 30, 1)
    p = oracle.resolve(f, 3.0, 20.0, 0.01, spatial="box")
    assert p.R == 3
    with pytest.raises(ValueError):
        oracle.box_radius(2.5)
    with pytest.raises(ValueError):
        oracle.box_radius(0.0)


def test_t_over_the_box_window():
    """Eq. (bound) with the box as the neighbourhood: T is the largest
    difference between a pixel and any pixel of its (2R+1)^2 square."""
    f = small_image(17, 13, 2)
    R = 2
    p = oracle.resolve(f, float(R), 20.0, 0.01, spatial="box")
    H, W = f.shape
    best = 0.0
    for y in range(H):
        for x in range(W):
            win = f[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1]
            best = max(best, float(np.max(np.abs(win - f[y, x]))))
    assert p.T[0, 0] == np.float32(best)


@pytest.mark.parametrize("shape,R", [((31, 40), 2), ((20, 9), 5), ((7, 50), 3)])
def test_large_sigma_r_is_box_mean(shape, R):
    """sigma_r -> infinity: the range kernel tends to 1 and the filter becomes
    the box mean over the clipped square (integral image)."""
    f = small_image(*shape, seed=R)
    sr = 1e6
    p = oracle.resolve(f, float(R), sr, 0.0, t_mode="fixed", t_fixed=255.0, spatial="box")
    out = oracle.shiftable(f, float(R), sr, p, spatial="box")
    ref = box_mean_integral(f, R)
    assert np.max(np.abs(out - ref)) < 1e-4
    dg = oracle.direct(f, float(R), sr, gauss=True, spatial="box")
    assert np.max(np.abs(dg - ref)) < 1e-4


@pytest.mark.parametrize("H,W,R,sr,eps,mode", [
    (9, 11, 1, 20.0, 0.0, "global"),
    (10, 8, 2, 12.0, 0.01, "global"),
    (12, 7, 3, 30.0, 0.05, "tile"),
])
def test_phi_filter_brute_force(H, W, R, sr, eps, mode):
    """Eq. (BF) with the box and phi_eps as the range kernel, summed pixel by
    pixel in Python, equals the oracle's shiftable box filter."""
    f = small_image(H, W, seed=H + W + R)
    p = oracle.resolve(f, float(R), sr, eps, t_mode=mode, t_tile=8, spatial="box")
    out = oracle.shiftable(f, float(R), sr, p, spatial="box")
    ref = np.empty_like(f)
    for y in range(H):
        for x in range(W):
            a, b = y // p.tile_h, x // p.tile_w
            N, M = int(p.N[a, b]), int(p.M[a, b])
            win = f[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1]
            w = phi_brute(win - f[y, x], N, M, sr)
            ref[y, x] = np.sum(w * win) / np.sum(w)
    assert np.max(np.abs(out - ref)) < 1e-9


def test_gaussian_range_brute_force():
    """The direct bilateral filter with the box and the Gaussian range kernel
    (eq. (BF)), summed in Python, equals the oracle's direct form."""
    f = small_image(12, 11, 6)
    R, sr = 2, 25.0
    got = oracle.direct(f, float(R), sr, gauss=True, spatial="box")
    H, W = f.shape
    ref = np.empty_like(f)
    for y in range(H):
        for x in range(W):
            win = f[max(0, y - R):y + R + 1, max(0, x - R):x + R + 1]
            w = np.exp(-(win - f[y, x]) ** 2 / (2 * sr * sr))
            ref[y, x] = np.sum(w * win) / np.sum(w)
    assert np.max(np.abs(got - ref)) < 1e-10


@pytest.mark.parametrize("H,W,R,sr,eps,mode,rule,tile", [
    (16, 16, 1, 20.0, 0.0, "fixed", "alg2", 64),
    (23, 37, 3, 8.0, 0.01, "global", "chernoff", 64),
    (40, 17, 4, 30.0, 0.05, "tile", "trunc", 16),
])
def test_shiftable_equals_direct(H, W, R, sr, eps, mode, rule, tile):
    """Sec. 1.2 with the box: modulate, box-filter, demodulate equals the
    direct phi_eps sum to rounding."""
    f = small_image(H, W, seed=H * 31 + W)
    p = oracle.resolve(f, float(R), sr, eps, t_mode=mode, rule=rule, t_tile=tile,
                       t_fixed=255.0 if mode == "fixed" else None, spatial="box")
    a, num_a, den_a, _ = oracle.shiftable(f, float(R), sr, p, return_parts=True, spatial="box")
    b, num_b, den_b, _ = oracle.direct(f, float(R), sr, p, return_parts=True, spatial="box")
    assert np.max(np.abs(den_a - den_b) / np.abs(den_b).max()) < 1e-10
    assert np.max(np.abs(num_a - num_b) / np.abs(num_b).max()) < 1e-10
    assert np.max(np.abs(a - b)) < 1e-8 * 255


def test_constant_image_and_shift():
    """A constant image passes unchanged (T = 0, N = 1), and the filter
    commutes with f -> f + c."""
    f = np.full((11, 14), 42.5)
    p = oracle.resolve(f, 3.0, 10.0, 0.01, spatial="box")
    assert float(p.T[0, 0]) == 0.0 and int(p.N[0, 0]) == 1
    assert np.max(np.abs(oracle.shiftable(f, 3.0, 10.0, p, spatial="box") - 42.5)) < 1e-12
    g = small_image(15, 12, 9)
    pg = oracle.resolve(g, 2.0, 20.0, 0.01, t_mode="fixed", t_fixed=255.0, spatial="box")
    a = oracle.shiftable(g, 2.0, 20.0, pg, spatial="box")
    b = oracle.shiftable(g + 17.0, 2.0, 20.0, pg, spatial="box")
    assert np.max(np.abs(b - a - 17.0)) < 1e-9


def test_gradient_forms_and_fd():
    """Gradient of L = sum u * out with the box (T, N, M fixed): shiftable
    form, direct form and central differences (h = 1e-3, FP64) agree."""
    f = small_image(13, 15, 8)
    R, sr, eps = 2, 25.0, 0.01
    p = oracle.resolve(f, float(R), sr, eps, spatial="box")
    u = np.random.default_rng(5).normal(size=f.shape)
    gs = oracle.grad_shiftable(f, u, float(R), sr, p, spatial="box")
    gd = oracle.grad_direct(f, u, float(R), sr, p, spatial="box")
    scale = np.max(np.abs(gd))
    assert np.max(np.abs(gs - gd)) < 1e-9 * scale
    h = 1e-3
    rng = np.random.default_rng(6)
    for _ in range(6):
        i, j = rng.integers(0, 13), rng.integers(0, 15)
        fp, fm = f.copy(), f.copy()
        fp[i, j] += h
        fm[i, j] -= h
        fd = (np.sum(u * oracle.shiftable(fp, float(R), sr, p, spatial="box")) -
              np.sum(u * oracle.shiftable(fm, float(R), sr, p, spatial="box"))) / (2 * h)
        assert abs(fd - gs[i, j]) < 1e-6 * scale + 1e-6 * abs(fd)
