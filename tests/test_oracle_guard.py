"""Pin of the oracle's denominator guard (reading of Sec. 3, where the paper
is silent): where den(x) <= 1e-6 * (g * 1_Omega)(x), the clipped spatial
mass at x, the output is f(x).

phi_eps of eq. (approx) drops binomial tails of total weight <= eps, so it
dips below zero (down to about -eps) away from s = 0.  A single outlier of
height A in a flat field then has

    den(x0) = g(0)^2 phi_eps(0) + (m(x0) - g(0)^2) phi_eps(A),

m(x0) the clipped mass, which is negative for a suitable A, while every
other pixel keeps den > 0.  The expected den, num and mass below are
computed here in plain Python (math.comb weights, math.cos, math.exp taps)
on the direct sum of eq. (BF), independent of the oracle's code; A is
tuned by bisection so that den / m lands on either side of the threshold.
The outliers sit at the image border, where m is the clipped mass (about a
third of the full window's), so a guard using the full mass, or another
threshold, or another fallback value fails one of the cases.
"""
import math

import numpy as np
import pytest

import oracle

SS, SR, EPS, T = 3.0, 10.0, 0.2, 80.0
R = 9          # ceil(3 sigma_s)


def taps_py():
    return [math.exp(-k * k / (2.0 * SS * SS)) for k in range(-R, R + 1)]


def mass_py(i, j, H, W):
    g = taps_py()
    sy = sum(g[a - i + R] for a in range(max(0, i - R), min(H - 1, i + R) + 1))
    sx = sum(g[b - j + R] for b in range(max(0, j - R), min(W - 1, j + R) + 1))
    return sy * sx


def nm_py():
    """N by Sec. 1.3 and M by eq. (trunc), in exact integer arithmetic."""
    N = math.ceil(4.0 * T * T / (math.pi ** 2 * SR * SR))
    # smallest M with sum_{n <= M+1} C(N, n) / 2^N > eps / 2
    M, S = 0, math.comb(N, 0)
    while True:
        S += math.comb(N, M + 1)
        if S / 2 ** N > EPS / 2:
            break
        M += 1
    return N, min(M, N // 2)


def phi_py(s, N, M):
    sc = math.sqrt(N) * SR
    return math.fsum(math.comb(N, n) / 2 ** N * math.cos((2 * n - N) * s / sc)
                     for n in range(M, N - M + 1))


def direct_py(f, i, j, N, M):
    """num and den of eq. (BF) at (i, j) with phi_eps, clipped window."""
    H, W = f.shape
    g = taps_py()
    num, den = [], []
    for a in range(max(0, i - R), min(H - 1, i + R) + 1):
        for b in range(max(0, j - R), min(W - 1, j + R) + 1):
            w = g[a - i + R] * g[b - j + R] * phi_py(f[a, b] - f[i, j], N, M)
            num.append(w * f[a, b])
            den.append(w)
    return math.fsum(num), math.fsum(den)


def outlier_height(ratio, i, j, H, W, N, M):
    """A in (0, A_min] with den(x0) / m(x0) = ratio for an outlier of height
    A at (i, j) in a zero field (den decreases in A up to phi_eps's dip)."""
    m = mass_py(i, j, H, W)
    p0 = phi_py(0.0, N, M)

    def den_over_m(A):
        return (p0 + (m - 1.0) * phi_py(A, N, M)) / m

    grid = np.linspace(0.0, T, 4001)
    vals = [den_over_m(a) for a in grid]
    hi = grid[int(np.argmin(vals))]
    assert den_over_m(hi) < ratio, "ratio not reachable at this position"
    lo = 0.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if den_over_m(mid) > ratio:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def resolve(f):
    p = oracle.resolve(f, SS, SR, EPS, t_mode="fixed", t_fixed=T, rule="trunc")
    N, M = nm_py()
    assert (p.N[0, 0], p.M[0, 0]) == (N, M)
    return p, N, M


# (row, column, target den / mass, fires): border and corner positions
CASES = [
    (1, 0, 1.2e-6, False),    # just above the threshold (with the full mass it would fire)
    (1, 0, 0.7e-6, True),     # just below it
    (0, 6, 1.3e-6, False),    # top row: the row sum of the mass is clipped
    (0, 6, 0.3e-6, True),
    (6, 0, 1.3e-6, False),    # left column: the column sum is clipped
    (1, 1, -0.005, True),     # clearly negative
    (4, 0, 0.02, False),      # clearly positive
]


@pytest.mark.parametrize("i,j,ratio,fires", CASES)
@pytest.mark.parametrize("form", ["shiftable", "direct"])
def test_guard_threshold_mass_and_fallback(i, j, ratio, fires, form):
    H, W = 24, 20
    N, M = nm_py()
    A = outlier_height(ratio, i, j, H, W, N, M)
    f = np.zeros((H, W))
    f[i, j] = A
    p, _, _ = resolve(f)
    num_e, den_e = direct_py(f, i, j, N, M)
    m = mass_py(i, j, H, W)
    assert abs(den_e / m - ratio) < 1e-3 * abs(ratio)
    assert (den_e <= 1e-6 * m) == fires
    if form == "shiftable":
        out, num, den, nfb = oracle.shiftable(f, SS, SR, p, return_parts=True)
        o, n_, d_ = out[i, j], num[i, j], den[i, j]
    else:
        out, num, den, nfb = oracle.direct(f, SS, SR, p, points=([i], [j]), return_parts=True)
        o, n_, d_ = out[0], num[0], den[0]
    # the oracle's sums are those of eq. (BF) with phi_eps
    assert abs(d_ - den_e) <= 1e-11 * m
    assert abs(n_ - num_e) <= 1e-11 * m * A
    if fires:
        assert o == A                      # f(x0), exactly
    else:
        assert abs(o - num_e / den_e) <= 1e-5 * abs(num_e / den_e)
    if form == "direct":
        assert nfb == (1 if fires else 0)


@pytest.mark.parametrize("form", ["shiftable", "direct"])
def test_guard_count_over_an_image(form):
    """Several outliers in one image, some past the threshold and some not:
    the oracle's count of guarded outputs (nfb) is the number of pixels whose
    independent den is <= 1e-6 of their clipped mass, and those outputs are
    f(x) exactly.  Outliers are far enough apart (> 2R) not to see each
    other, and every other pixel's den is positive."""
    H, W = 60, 80
    N, M = nm_py()
    spots = [(1, 0, 0.3e-6), (0, 30, 0.5e-6), (59, 78, 5e-6), (30, 79, -0.002),
             (59, 40, 0.02), (1, 60, -0.005)]
    f = np.zeros((H, W))
    for i, j, ratio in spots:
        f[i, j] = outlier_height(ratio, i, j, H, W, N, M)
    for a in range(len(spots)):
        for b in range(a + 1, len(spots)):
            (i1, j1, _), (i2, j2, _) = spots[a], spots[b]
            assert max(abs(i1 - i2), abs(j1 - j2)) > 2 * R
    p, _, _ = resolve(f)
    fired = []
    for i, j, _ in spots:
        num_e, den_e = direct_py(f, i, j, N, M)
        if den_e <= 1e-6 * mass_py(i, j, H, W):
            fired.append((i, j))
    assert 0 < len(fired) < len(spots)
    if form == "shiftable":
        out, num, den, nfb = oracle.shiftable(f, SS, SR, p, return_parts=True)
    else:
        out, num, den, nfb = oracle.direct(f, SS, SR, p, return_parts=True)
    assert nfb == len(fired)
    for i, j in fired:
        assert out[i, j] == f[i, j]
    # every other output is a weighted mean of its window (no fallback)
    mask = np.ones_like(f, dtype=bool)
    for i, j in fired:
        mask[i, j] = False
    assert np.all(den[mask] > 0)
