"""Pins of the oracle's non-local means with a p-pixel patch (Sec. 6, eqs.
(NL1), (NL2)): a multivariate range kernel, the product over the patch
pixels u_1 = 0, u_2, ..., u_p of one-dimensional raised-cosine kernels
phi_eps with the N, M of T (eq. (bound), Algorithm 1), and its O(1)
shiftable form (one pair of modulated planes per multi-index of the product
expansion; N^p terms, the count Sec. 6 points out).

Pinned by: the one-pixel patch reducing to the bilateral filter (the oracle's
own, independently pinned, direct form); brute force in pure Python (with
exact binomial weights and math.cos, and with the exact Gaussian product,
i.e. the textbook patch-distance weight); the shiftable expansion agreeing
with the direct sums; T covering every patch difference; invariants.
Patch values outside the image are taken at the nearest in-image pixel.
"""
from math import comb, cos, exp, sqrt

import numpy as np
import pytest

import oracle
from paper_1203_5128_gb300 import synth

CENTRE, RIGHT, DOWN, LEFT, UP = 1 << 4, 1 << 5, 1 << 7, 1 << 3, 1 << 1
P3 = CENTRE | RIGHT | DOWN
P5 = CENTRE | RIGHT | DOWN | LEFT | UP


def test_patch_offsets():
    uy, ux = oracle.patch_offsets(P3)
    assert list(zip(uy, ux)) == [(0, 0), (0, 1), (1, 0)]
    uy, ux = oracle.patch_offsets(0x1FF)
    assert len(uy) == 9 and (uy[0], ux[0]) == (0, 0)
    with pytest.raises(ValueError):
        oracle.patch_offsets(RIGHT)


@pytest.mark.parametrize("spatial,ss", [("box", 2.0), ("fir", 1.3)])
def test_one_pixel_patch_is_the_bilateral_filter(spatial, ss):
    f = synth.g8(23, 19, seed=7).astype(np.float64)
    p = oracle.resolve(f, ss, 25.0, 0.02, t_mode="global", rule="trunc", spatial=spatial)
    a = oracle.nlm_direct(f, ss, 25.0, p, CENTRE, spatial=spatial)
    b = oracle.direct(f, ss, 25.0, p, spatial=spatial)
    assert np.max(np.abs(a - b)) < 1e-11


def clamp_f(f, y, x):
    H, W = f.shape
    return f[min(max(y, 0), H - 1), min(max(x, 0), W - 1)]


def brute_nlm(f, R, sigma_r, N, M, offs, gauss):
    """eqs. (NL1) / (NL2) with the box window, pure Python."""
    H, W = f.shape
    w = [comb(N, n) / 2 ** N for n in range(N + 1)]
    om = [(2 * n - N) / (sqrt(N) * sigma_r) for n in range(N + 1)]

    def phi(s):
        if gauss:
            return exp(-s * s / (2 * sigma_r * sigma_r))
        return sum(w[n] * cos(om[n] * s) for n in range(M, N - M + 1))
    out = np.empty_like(f)
    for i in range(H):
        for j in range(W):
            num = den = 0.0
            for a in range(max(0, i - R), min(H, i + R + 1)):
                for b in range(max(0, j - R), min(W, j + R + 1)):
                    k = 1.0
                    for dy, dx in offs:
                        k *= phi(clamp_f(f, i + dy, j + dx) - clamp_f(f, a + dy, b + dx))
                    num += k * f[a, b]
                    den += k
            out[i, j] = num / den
    return out


@pytest.mark.parametrize("mask,gauss", [(P3, False), (P5, False), (P3, True)])
def test_nlm_direct_matches_brute_force(mask, gauss):
    f = synth.g8(9, 11, seed=3).astype(np.float64)
    R, sr = 2, 40.0
    p = oracle.resolve(f, float(R), sr, 0.05, t_mode="global", rule="trunc", spatial="box")
    uy, ux = oracle.patch_offsets(mask)
    out = oracle.nlm_direct(f, float(R), sr, p, mask, gauss=gauss, spatial="box")
    ref = brute_nlm(f, R, sr, int(p.N[0, 0]), int(p.M[0, 0]), list(zip(uy, ux)), gauss)
    assert np.max(np.abs(out - ref)) < 1e-10


@pytest.mark.parametrize("mask,spatial,eps", [(P3, "box", 0.05), (CENTRE | RIGHT, "fir", 0.0),
                                              (P3, "fir", 0.02)])
def test_nlm_shiftable_equals_direct(mask, spatial, eps):
    """Sec. 6: the product of the per-pixel expansions gives the O(1) form;
    it reproduces the direct sums to rounding."""
    f = synth.g8(18, 21, seed=5).astype(np.float64)
    ss, sr = 2.0, 45.0
    p = oracle.resolve(f, ss, sr, eps, t_mode="global", rule="trunc", spatial=spatial)
    a, _, da, _ = oracle.nlm_shiftable(f, ss, sr, p, mask, spatial=spatial, return_parts=True)
    b, _, db, _ = oracle.nlm_direct(f, ss, sr, p, mask, spatial=spatial, return_parts=True)
    assert np.max(np.abs(da - db)) < 1e-10 * np.max(np.abs(db))
    assert np.max(np.abs(a - b)) < 1e-9


def test_t_covers_every_patch_difference():
    """Sec. 6: every component s_i = f(x + u_i) - f(x - y + u_i) lies in
    [-T, T] with T of eq. (bound) (both pixels are within R of each other,
    also after clamping to the image), so the one-dimensional kernels need
    the raised cosine on [-T, T] only."""
    f = synth.g8(21, 17, seed=8).astype(np.float64)
    R = 3
    T = float(oracle.t_global(f, R))
    uy, ux = oracle.patch_offsets(0x1FF)
    H, W = f.shape
    worst = 0.0
    for i in range(H):
        for j in range(W):
            for a in range(max(0, i - R), min(H, i + R + 1)):
                for b in range(max(0, j - R), min(W, j + R + 1)):
                    for dy, dx in zip(uy, ux):
                        worst = max(worst, abs(clamp_f(f, i + dy, j + dx) -
                                               clamp_f(f, a + dy, b + dx)))
    assert worst <= T


def test_nlm_constant_image_and_large_sigma_r():
    f = np.full((10, 13), 42.0)
    p = oracle.resolve(f, 2.0, 30.0, 0.01, t_mode="global", spatial="box")
    assert np.max(np.abs(oracle.nlm_direct(f, 2.0, 30.0, p, P5) - 42.0)) < 1e-12
    g = synth.g8(12, 15, seed=2).astype(np.float64)
    pg = oracle.resolve(g, 2.0, 1e7, 0.0, t_mode="fixed", t_fixed=255.0, spatial="box")
    out = oracle.nlm_direct(g, 2.0, 1e7, pg, P3)
    # box mean over the clipped window
    H, W = g.shape
    ref = np.empty_like(g)
    for i in range(H):
        for j in range(W):
            ref[i, j] = g[max(0, i - 2):i + 3, max(0, j - 2):j + 3].mean()
    assert np.max(np.abs(out - ref)) < 1e-6


def test_nlm_transpose():
    """Transposing the image and the patch transposes the output."""
    f = synth.g8(14, 17, seed=6).astype(np.float64)
    p = oracle.resolve(f, 2.0, 35.0, 0.02, t_mode="global", rule="trunc", spatial="box")
    a = oracle.nlm_direct(f, 2.0, 35.0, p, CENTRE | RIGHT)
    pt = oracle.resolve(f.T.copy(), 2.0, 35.0, 0.02, t_mode="global", rule="trunc", spatial="box")
    b = oracle.nlm_direct(f.T.copy(), 2.0, 35.0, pt, CENTRE | DOWN)
    assert np.max(np.abs(a.T - b)) < 1e-11
