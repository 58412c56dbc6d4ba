"""Pins of the oracle's raised-polynomial range kernel (Sec. 1.3, eqs. (RP)
and (RPconv)): phi(s) = (1 - s^2 / (2 N sigma_r^2))^N with N = max(1,
ceil(T^2 / (2 sigma_r^2))), the filter of eq. (BF) with it as range kernel,
and the T it is taken with (the range of f over each T-tile grown by R).

None of these retypes the oracle's formula: they use the Gaussian limit of
eq. (RPconv), the positivity / monotonicity threshold N0 = 0.5 (T /
sigma_r)^2 the paper states, the root of the kernel, exact rational
binomial sums, brute force in pure Python, invariants (shift, scale,
constant image, sigma_r -> infinity), and the shiftability of the kernel in
a polynomial basis (eqs. (f1), (f2)) checked in exact rational arithmetic.
"""
from fractions import Fraction
from math import comb, exp, sqrt

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_1203_5128_gb300 import synth


def test_rp_gaussian_limit():
    """eq. (RPconv): (1 - s^2/(2 N sigma^2))^N -> exp(-s^2/(2 sigma^2)); the
    sup error on [-T, T] falls with N, roughly like 1/N."""
    sr, T = 20.0, 255.0
    s = np.linspace(-T, T, 4001)
    g = np.exp(-s ** 2 / (2 * sr ** 2))
    Ns = [82, 164, 328, 656, 1312]
    errs = [float(np.max(np.abs(oracle.poly_phi(s, N, sr) - g))) for N in Ns]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    for N, e in zip(Ns, errs):
        assert e * N < 1.0
    assert errs[-1] < 5e-4


@pytest.mark.parametrize("T,sr", [(255.0, 30.0), (255.0, 20.0), (100.0, 7.0), (65535.0, 5000.0),
                                  (37.5, 11.0)])
def test_rp_positive_monotone_from_n0(T, sr):
    """Sec. 1.3: the argument of eq. (RPconv) stays in [0, 1] on [-T, T] (so
    phi is positive and non-increasing in |s|) once N >= 0.5 (T / sigma_r)^2;
    the order the oracle picks is the smallest such integer (>= 1).  With
    one order less the kernel's root sqrt(2 (N-1)) sigma_r falls inside
    (0, T): phi vanishes there and is not positive on [-T, T]."""
    N = oracle.poly_order(T, sr)
    n0 = 0.5 * (T / sr) ** 2
    assert N == max(1, int(np.ceil(n0 - 1e-12)))
    s = np.linspace(0.0, T, 20001)
    p = oracle.poly_phi(s, N, sr)
    assert np.all(p >= 0.0) and np.all(np.diff(p) <= 1e-15)
    assert sqrt(2 * N) * sr >= T
    if N > 1 and N - 1 < n0:
        root = sqrt(2 * (N - 1)) * sr
        assert root < T and abs(oracle.poly_phi(root, N - 1, sr)[0]) < 1e-12


@pytest.mark.parametrize("N", [1, 4, 37, 500])
def test_rp_root_and_peak(N):
    """phi(0) = 1, and phi vanishes (a root of order N) at s = sqrt(2 N) sigma_r."""
    sr = 13.0
    assert oracle.poly_phi(0.0, N, sr)[0] == 1.0
    assert abs(oracle.poly_phi(sqrt(2 * N) * sr, N, sr)[0]) < 1e-12


def test_rp_binomial_expansion_exact():
    """The kernel equals its binomial expansion sum_k C(N, k) (-s^2/a)^k,
    a = 2 N sigma_r^2, evaluated exactly in rationals."""
    sr = Fraction(25)
    for N in [3, 11, 40]:
        a = 2 * N * sr * sr
        for s in [Fraction(0), Fraction(7, 2), Fraction(61), Fraction(123, 3), Fraction(200)]:
            exact = sum(comb(N, k) * (-s * s / a) ** k for k in range(N + 1))
            got = oracle.poly_phi(float(s), N, float(sr))[0]
            assert abs(got - float(exact)) <= 1e-12 * max(1.0, abs(float(exact)))


def test_rp_range_tiles_brute():
    """T per tile: max - min of f over the tile grown by R, clipped."""
    f = synth.g8(37, 53, seed=4).astype(np.float64)
    for R, th, tw in [(3, 8, 8), (5, 16, 32), (0, 37, 53), (40, 64, 64)]:
        T = oracle.range_tiles(f, R, th, tw)
        for a in range(T.shape[0]):
            for b in range(T.shape[1]):
                blk = f[max(0, a * th - R):(a + 1) * th + R, max(0, b * tw - R):(b + 1) * tw + R]
                assert T[a, b] == blk.max() - blk.min()


def brute_poly(f, sigma_s, sigma_r, N_of, R):
    """eq. (BF) with the raised polynomial, pure Python loops."""
    H, W = f.shape
    g = [exp(-k * k / (2.0 * sigma_s * sigma_s)) for k in range(-R, R + 1)]
    out = np.empty_like(f)
    for i in range(H):
        for j in range(W):
            N = N_of(i, j)
            a = 2.0 * N * sigma_r * sigma_r
            num = den = 0.0
            for y in range(max(0, i - R), min(H, i + R + 1)):
                for x in range(max(0, j - R), min(W, j + R + 1)):
                    s = f[y, x] - f[i, j]
                    w = g[y - i + R] * g[x - j + R] * (1.0 - s * s / a) ** N
                    num += w * f[y, x]
                    den += w
            out[i, j] = num / den
    return out


@pytest.mark.parametrize("mode,tile", [("fixed", 64), ("global", 64), ("tile", 8)])
def test_rp_direct_matches_brute_force(mode, tile):
    f = synth.g8(16, 18, seed=9).astype(np.float64)
    ss, sr = 1.4, 30.0
    p = oracle.resolve(f, ss, sr, t_mode=mode, t_tile=tile, t_fixed=255.0, kernel="poly")
    assert np.all(p.M == 0)
    out = oracle.poly_direct(f, ss, sr, p)
    th, tw = min(p.tile_h, 1 << 20), min(p.tile_w, 1 << 20)
    ref = brute_poly(f, ss, sr, lambda i, j: int(p.N[i // th, j // tw]), p.R)
    assert np.max(np.abs(out - ref)) < 1e-10


def test_rp_constant_image():
    f = np.full((11, 17), 91.5)
    p = oracle.resolve(f, 2.0, 10.0, t_mode="tile", t_tile=8, kernel="poly")
    assert np.all(p.T == 0.0) and np.all(p.N == 1)
    assert np.max(np.abs(oracle.poly_direct(f, 2.0, 10.0, p) - 91.5)) < 1e-12


def test_rp_large_sigma_r_is_normalised_blur():
    """sigma_r -> infinity: the kernel tends to 1, eq. (BF) to the clipped
    normalised Gaussian blur (scipy.ndimage, zero padding)."""
    f = synth.g8(23, 31, seed=3).astype(np.float64)
    ss, sr = 1.7, 1e7
    p = oracle.resolve(f, ss, sr, t_mode="fixed", t_fixed=255.0, kernel="poly")
    out = oracle.poly_direct(f, ss, sr, p)
    R = oracle.radius(ss)
    k = np.exp(-np.arange(-R, R + 1) ** 2 / (2 * ss ** 2))

    def blur(x):
        x = ndimage.correlate1d(x, k, axis=1, mode="constant", cval=0.0)
        return ndimage.correlate1d(x, k, axis=0, mode="constant", cval=0.0)
    assert np.max(np.abs(out - blur(f) / blur(np.ones_like(f)))) < 1e-6


def test_rp_shift_and_scale_covariance():
    """f -> f + c leaves every range (so T and N) unchanged and shifts the
    output; (f, sigma_r) -> (a f, a sigma_r) scales T by a, keeps N and
    scales the output."""
    f = synth.g8(19, 23, seed=11).astype(np.float64)
    ss, sr = 1.5, 28.0
    p = oracle.resolve(f, ss, sr, t_mode="tile", t_tile=8, kernel="poly")
    base = oracle.poly_direct(f, ss, sr, p)
    p1 = oracle.resolve(f + 500.0, ss, sr, t_mode="tile", t_tile=8, kernel="poly")
    assert np.array_equal(p1.N, p.N)
    assert np.max(np.abs(oracle.poly_direct(f + 500.0, ss, sr, p1) - 500.0 - base)) < 1e-8
    a = 4.0
    p2 = oracle.resolve(a * f, ss, a * sr, t_mode="tile", t_tile=8, kernel="poly")
    assert np.array_equal(p2.N, p.N)
    assert np.max(np.abs(oracle.poly_direct(a * f, ss, a * sr, p2) / a - base)) < 1e-9


def test_rp_kernel_is_shiftable_in_a_polynomial_basis():
    """eqs. (f1), (f2) with basis phi_j(s) = s^j: (1 - (s - t)^2 / a)^N =
    sum_j c_j(t) s^j, so num = sum_j c_j(f(x)) (g * f^{j+1})(x) and den =
    sum_j c_j(f(x)) (g * f^j)(x).  Evaluated exactly in rationals on a tiny
    image with integer values and a box spatial kernel, it equals the
    oracle's direct sum at every pixel."""
    rng = np.random.default_rng(2)
    f = rng.integers(0, 40, size=(6, 7)).astype(np.float64)
    R, sr = 1, 9.0
    p = oracle.resolve(f, 1.0, sr, t_mode="global", kernel="poly", spatial="box")
    N = int(p.N[0, 0])
    a = Fraction(2 * N) * Fraction(sr) ** 2
    H, W = f.shape
    # c_j(t) from (1 - (s - t)^2 / a)^N = sum_k C(N,k) (-1/a)^k sum_j C(2k,j) s^j (-t)^(2k-j)
    def coeffs(t):
        c = [Fraction(0)] * (2 * N + 1)
        for k in range(N + 1):
            ck = comb(N, k) * Fraction(-1) ** k / a ** k
            for j in range(2 * k + 1):
                c[j] += ck * comb(2 * k, j) * (-t) ** (2 * k - j)
        return c
    out = oracle.poly_direct(f, 1.0, sr, p, spatial="box")
    for i in range(H):
        for j in range(W):
            t = Fraction(int(f[i, j]))
            c = coeffs(t)
            num = den = Fraction(0)
            for y in range(max(0, i - R), min(H, i + R + 1)):
                for x in range(max(0, j - R), min(W, j + R + 1)):
                    v = Fraction(int(f[y, x]))
                    pw = Fraction(1)
                    for q in range(2 * N + 1):
                        den += c[q] * pw
                        num += c[q] * pw * v
                        pw *= v
            assert abs(out[i, j] - float(num / den)) < 1e-9
