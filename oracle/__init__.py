"""FP64 CPU oracle for the shiftable bilateral filter (arXiv:1203.5128).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA path and never imports it.

The arithmetic lives in ``bf_oracle.c`` (plain double-precision C, one
routine per step of the paper); this module only marshals numpy arrays and
strings the steps together in the order of Algorithm 2:

1. R = ceil(3 sigma_s)                                   (Sec. 2)
2. T from the windowed max/min filter                    (eq. (bound), Alg. 1)
3. N = max(1, ceil(4 T^2 / (pi^2 sigma_r^2)))            (Sec. 1.3)
4. M by eq. (trunc), eq. (Chernoff) or the Alg. 2 bands  (Sec. 3)
5. phi_eps with weights 2^-N C(N, n), n = M..N-M         (eq. (approx))
6. SHIFTABLE-BF with phi_eps                             (Sec. 1.2)

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, brute force, exact rational arithmetic and the
values the paper prints).  The denominator guard (where den <= 1e-6 of the
clipped spatial mass the output is f(x); the paper is silent) and the
clipped mass it uses are pinned by ``tests/test_oracle_guard.py`` against
den, num and mass computed in plain Python at outliers tuned to either
side of the threshold at the image border.  The Young-van Vliet mode (``spatial="yvv"``) is
pinned by ``tests/test_oracle_yvv.py`` against the recursion's closed-form
frequency response, brute-force convolution with its impulse response and
the direct form; the paper prints no value for it.  The box mode
(``spatial="box"``: the constant spatial filter of radius sigma_s that
Sec. 4 uses against BF2) is pinned by ``tests/test_oracle_box.py`` against
running sums of an integral image, pure-Python brute force and the direct
form.  The raised-polynomial kernel (``resolve(..., kernel="poly")``,
``poly_direct``: Sec. 1.3, eqs. (RP), (RPconv)) is pinned by
``tests/test_oracle_poly.py``: its Gaussian limit, positivity and
monotonicity from N0 on, the binomial expansion in exact arithmetic, the
region ranges and the direct sum by pure-Python brute force, the constant
image, the sigma_r -> infinity blur, covariance and shiftability in a
polynomial basis.  The non-local means (``nlm_direct``, ``nlm_shiftable``:
Sec. 6, eqs. (NL1), (NL2)) are pinned by ``tests/test_oracle_nlm.py``: the
one-pixel patch is the bilateral filter, the direct sum equals pure-Python
brute force (raised cosine and exact Gaussian), the shiftable form equals
the direct sum, T covers every patch difference, the constant image and
large sigma_r, transposition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Threshold-mode and truncation-rule names shared with the tests (strings,
# so that nothing numeric is shared with the CUDA path).
T_FIXED, T_GLOBAL, T_TILE = "fixed", "global", "tile"
RULE_ALG2, RULE_TRUNC, RULE_CHERNOFF = "alg2", "trunc", "chernoff"
WHOLE = 1 << 30          # tile extent of a single-kernel (fixed / global T) plan


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (-O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    D, I, L = ctypes.c_double, ctypes.c_int, ctypes.c_long
    P = ctypes.c_void_p
    sig = {
        "orc_num_threads": (I, []),
        "orc_radius": (I, [D]),
        "orc_gauss_taps": (None, [D, I, P]),
        "orc_maxmin_brute": (None, [P, I, I, I, P, P]),
        "orc_maxmin_vhgw": (L, [P, I, I, I, P, P]),
        "orc_local_range": (None, [P, P, P, I, I, P]),
        "orc_t_tiles": (None, [P, I, I, I, I, P]),
        "orc_n0": (D, [D, D]),
        "orc_order": (I, [D, D]),
        "orc_log_weights": (None, [I, P]),
        "orc_trunc_m": (I, [I, D]),
        "orc_chernoff_m": (I, [I, D]),
        "orc_alg2_m": (I, [I, D, D, D]),
        "orc_phi_eval": (None, [P, I, I, I, D, P]),
        "orc_shiftable_block": (L, [P, I, I, P, I, I, I, D, I, I, I, I, P, P, P]),
        "orc_direct_points": (L, [P, I, I, P, I, P, P, D, I, P, P, I, P, P, P]),
        "orc_grad_shiftable_block": (None, [P, I, I, P, I, I, I, D, I, I, I, I, P, P, P]),
        "orc_grad_direct_points": (None, [P, I, I, P, I, I, I, D, P, P, P, P, I, P]),
        "orc_yvv_coeffs": (None, [D, P]),
        "orc_yvv_margin": (I, [D]),
        "orc_yvv_2d": (None, [P, P, I, I, D, I]),
        "orc_yvv_impulse": (None, [D, I, P]),
        "orc_shiftable_yvv": (L, [P, I, I, D, I, I, D, P, P, P]),
        "orc_poly_order": (I, [D, D]),
        "orc_poly_phi": (None, [P, I, I, D, P]),
        "orc_range_tiles": (None, [P, I, I, I, I, I, P]),
        "orc_poly_direct_points": (L, [P, I, I, P, I, P, D, P, P, I, P, P, P]),
        "orc_nlm_direct_points": (L, [P, I, I, P, I, I, I, D, I, P, P, I, P, P, I, P, P, P]),
        "orc_nlm_shiftable": (L, [P, I, I, P, I, I, I, D, P, P, I, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(f) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(f, dtype=np.float64))


def num_threads() -> int:
    return _load().orc_num_threads()


# ---------------------------------------------------------------- kernels

def radius(sigma_s: float) -> int:
    """R = ceil(3 sigma_s) (Sec. 2)."""
    return _load().orc_radius(float(sigma_s))


def taps(sigma_s: float, R: int | None = None) -> np.ndarray:
    """Spatial Gaussian taps g[k+R] = exp(-k^2/(2 sigma_s^2)), k=-R..R."""
    if R is None:
        R = radius(sigma_s)
    g = np.empty(2 * R + 1)
    _load().orc_gauss_taps(float(sigma_s), R, _p(g))
    return g


def box_radius(sigma_s: float) -> int:
    """Radius of the constant (box) spatial filter.  In the comparison with
    BF2 (Sec. 4, Figs. 7-10) sigma_s names the radius of the box, so it must
    be a positive integer; the window is the (2 sigma_s + 1)^2 square."""
    r = float(sigma_s)
    if not (r >= 1.0 and r == int(r)):
        raise ValueError("box radius sigma_s must be a positive integer, got %r" % sigma_s)
    return int(r)


def spatial_taps(sigma_s: float, R: int, spatial: str) -> np.ndarray:
    """One-dimensional taps of the separable spatial filter: the truncated
    Gaussian ("fir") or the constant filter ("box"), whose 2-D kernel is
    the product of the two lines'."""
    if spatial == "fir":
        return taps(sigma_s, R)
    if spatial == "box":
        return np.ones(2 * R + 1)
    raise ValueError(spatial)


# ---------------------------------------------------------------- max / min

def maxmin_brute(f, R: int):
    f = _f64(f)
    H, W = f.shape
    Mx, mn = np.empty_like(f), np.empty_like(f)
    _load().orc_maxmin_brute(_p(f), H, W, R, _p(Mx), _p(mn))
    return Mx, mn


def maxmin_vhgw(f, R: int):
    """Returns (M, m, ops): the van Herk / Gil-Werman filters and the number
    of max/min operations they took (Appendix)."""
    f = _f64(f)
    H, W = f.shape
    Mx, mn = np.empty_like(f), np.empty_like(f)
    ops = _load().orc_maxmin_vhgw(_p(f), H, W, R, _p(Mx), _p(mn))
    return Mx, mn, ops


def local_range(f, R: int) -> np.ndarray:
    f = _f64(f)
    Mx, mn, _ = maxmin_vhgw(f, R)
    r = np.empty_like(f)
    _load().orc_local_range(_p(f), _p(Mx), _p(mn), f.shape[0], f.shape[1], _p(r))
    return r


def t_tiles(f, R: int, tile_h: int, tile_w: int) -> np.ndarray:
    """T per tile (FP32), grid anchored at (0,0)."""
    f = _f64(f)
    H, W = f.shape
    r = local_range(f, R)
    ty, tx = -(-H // tile_h), -(-W // tile_w)
    T = np.empty((ty, tx), dtype=np.float32)
    _load().orc_t_tiles(_p(r), H, W, tile_h, tile_w, _p(T))
    return T


def t_global(f, R: int) -> np.float32:
    f = _f64(f)
    H, W = f.shape
    return t_tiles(f, R, H, W)[0, 0]


# ---------------------------------------------------------------- N, M, w

def n0(T: float, sigma_r: float) -> float:
    return _load().orc_n0(float(T), float(sigma_r))


def order(T: float, sigma_r: float) -> int:
    return _load().orc_order(float(T), float(sigma_r))


def log_weights(N: int) -> np.ndarray:
    lw = np.empty(N + 1)
    _load().orc_log_weights(N, _p(lw))
    return lw


def trunc_m(N: int, eps: float) -> int:
    return _load().orc_trunc_m(N, float(eps))


def chernoff_m(N: int, eps: float) -> int:
    return _load().orc_chernoff_m(N, float(eps))


def alg2_m(N: int, sigma_r: float, eps: float, value_range: float = 255.0) -> int:
    return _load().orc_alg2_m(N, float(sigma_r), float(eps), float(value_range))


def choose_m(N: int, sigma_r: float, eps: float, rule: str, value_range: float) -> int:
    if rule == RULE_ALG2:
        return alg2_m(N, sigma_r, eps, value_range)
    if rule == RULE_TRUNC:
        return trunc_m(N, eps)
    if rule == RULE_CHERNOFF:
        return chernoff_m(N, eps)
    raise ValueError(rule)


def phi(s, N: int, M: int, sigma_r: float) -> np.ndarray:
    """phi_eps(s) of eq. (approx); M = 0 gives eq. (expansion)."""
    s = _f64(np.atleast_1d(s))
    out = np.empty_like(s)
    _load().orc_phi_eval(_p(s), s.size, N, M, float(sigma_r), _p(out))
    return out


# ---------------------------------------------------------------- plan

@dataclass
class Params:
    """Resolved parameters: per-tile arrays (a 1x1 grid for a single T)."""
    R: int
    tile_h: int
    tile_w: int
    T: np.ndarray      # float32 [ty, tx]
    N: np.ndarray      # int [ty, tx]
    M: np.ndarray      # int [ty, tx]

    @property
    def K(self) -> np.ndarray:
        return self.N - 2 * self.M + 1


def resolve(f, sigma_s: float, sigma_r: float, eps: float = 0.0, *,
            t_mode: str = T_GLOBAL, rule: str = RULE_ALG2,
            value_range: float = 255.0, t_fixed: float | None = None,
            t_tile: int = 64, spatial: str = "fir", kernel: str = "cos") -> Params:
    """Algorithm 2, steps 1-4: R, T, N and M (per T-tile in ``tile`` mode).
    R is ceil(3 sigma_s) for the Gaussian (and its recursive form) and
    sigma_s itself for the box filter (``spatial="box"``).  ``kernel="poly"``
    takes the raised polynomial of eq. (RPconv): N = max(1, ceil(T^2 /
    (2 sigma_r^2))), no truncation (M = 0), and T the range of f over the
    image (``global``) or over each T-tile grown by R (``tile``)."""
    f = _f64(f)
    H, W = f.shape
    R = box_radius(sigma_s) if spatial == "box" else radius(sigma_s)
    if kernel == "poly":
        return _resolve_poly(f, R, sigma_r, t_mode, value_range, t_fixed, t_tile)
    if kernel != "cos":
        raise ValueError(kernel)
    if t_mode == T_FIXED:
        T = np.array([[np.float32(value_range if t_fixed is None else t_fixed)]], np.float32)
        th = tw = WHOLE
    elif t_mode == T_GLOBAL:
        T = t_tiles(f, R, H, W)
        th = tw = WHOLE
    elif t_mode == T_TILE:
        T = t_tiles(f, R, t_tile, t_tile)
        th, tw = t_tile, t_tile
    else:
        raise ValueError(t_mode)
    N = np.vectorize(lambda t: order(float(t), sigma_r), otypes=[np.int64])(T)
    M = np.vectorize(lambda n: choose_m(int(n), sigma_r, eps, rule, value_range),
                     otypes=[np.int64])(N)
    return Params(R=R, tile_h=th, tile_w=tw, T=T, N=N, M=M)


def poly_order(T: float, sigma_r: float) -> int:
    """N = max(1, ceil(T^2 / (2 sigma_r^2))) (Sec. 1.3, raised polynomial)."""
    return _load().orc_poly_order(float(T), float(sigma_r))


def poly_phi(s, N: int, sigma_r: float) -> np.ndarray:
    """(1 - s^2 / (2 N sigma_r^2))^N, eq. (RPconv)."""
    s = _f64(np.atleast_1d(s))
    out = np.empty_like(s)
    _load().orc_poly_phi(_p(s), s.size, int(N), float(sigma_r), _p(out))
    return out


def range_tiles(f, R: int, tile_h: int, tile_w: int) -> np.ndarray:
    """max - min of f over each tile grown by R (clipped), float64."""
    f = _f64(f)
    H, W = f.shape
    ty, tx = -(-H // tile_h), -(-W // tile_w)
    T = np.empty((ty, tx))
    _load().orc_range_tiles(_p(f), H, W, int(R), int(tile_h), int(tile_w), _p(T))
    return T


def _resolve_poly(f, R, sigma_r, t_mode, value_range, t_fixed, t_tile) -> Params:
    H, W = f.shape
    if t_mode == T_FIXED:
        T = np.array([[float(value_range if t_fixed is None else t_fixed)]])
        th = tw = WHOLE
    elif t_mode == T_GLOBAL:
        T = range_tiles(f, R, H, W)
        th = tw = WHOLE
    elif t_mode == T_TILE:
        T = range_tiles(f, R, t_tile, t_tile)
        th, tw = t_tile, t_tile
    else:
        raise ValueError(t_mode)
    N = np.vectorize(lambda t: poly_order(float(t), sigma_r), otypes=[np.int64])(T)
    return Params(R=R, tile_h=th, tile_w=tw, T=T.astype(np.float32), N=N,
                  M=np.zeros_like(N))


def poly_direct(f, sigma_s: float, sigma_r: float, params: Params, *, points=None,
                return_parts=False, spatial: str = "fir"):
    """Direct sum of eq. (BF) with the raised-polynomial range kernel of each
    point's T-tile order (eq. (RPconv)), at the given points (all pixels if
    None)."""
    f = _f64(f)
    H, W = f.shape
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = np.asarray(points[0]), np.asarray(points[1])
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    g = spatial_taps(sigma_s, params.R, spatial)
    a, b = _tile_of(params, ys, xs)
    Ns = np.ascontiguousarray(params.N[a, b], dtype=np.int32)
    out, num, den = np.empty(ys.size), np.empty(ys.size), np.empty(ys.size)
    nfb = _load().orc_poly_direct_points(_p(f), H, W, _p(g), params.R, _p(Ns), float(sigma_r),
                                         _p(ys), _p(xs), ys.size, _p(out), _p(num), _p(den))
    if points is None:
        out, num, den = out.reshape(H, W), num.reshape(H, W), den.reshape(H, W)
    if return_parts:
        return out, num, den, nfb
    return out


# ---------------------------------------------------------------- non-local means

def patch_offsets(mask: int):
    """Patch pixels u_1..u_p of the non-local means of Sec. 6 from a 9-bit
    mask over the 3 x 3 neighbourhood (bit 3 (dy + 1) + (dx + 1)); the centre
    bit must be set and comes first (u_1 = 0)."""
    mask = int(mask)
    if not (mask & (1 << 4)) or mask >> 9:
        raise ValueError("patch mask must hold the centre (bit 4) and fit 9 bits: %r" % mask)
    offs = [(0, 0)]
    for b in range(9):
        if b != 4 and mask & (1 << b):
            offs.append((b // 3 - 1, b % 3 - 1))
    uy = np.ascontiguousarray([o[0] for o in offs], dtype=np.int32)
    ux = np.ascontiguousarray([o[1] for o in offs], dtype=np.int32)
    return uy, ux


def nlm_direct(f, sigma_s: float, sigma_r: float, params: Params, patch_mask: int, *,
               points=None, gauss: bool = False, spatial: str = "box", return_parts=False):
    """Direct sums of eqs. (NL1), (NL2) (Sec. 6): the range kernel is the
    product over the patch pixels of phi_eps (one (N, M) for the image), or
    of exact Gaussians when ``gauss``; ``spatial`` "box" weighs the window
    equally (the paper's sums), "fir" with the Gaussian."""
    assert params.T.size == 1, "non-local means takes one (N, M)"
    f = _f64(f)
    H, W = f.shape
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = np.asarray(points[0]), np.asarray(points[1])
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    uy, ux = patch_offsets(patch_mask)
    g = spatial_taps(sigma_s, params.R, spatial)
    out, num, den = np.empty(ys.size), np.empty(ys.size), np.empty(ys.size)
    nfb = _load().orc_nlm_direct_points(_p(f), H, W, _p(g), params.R, int(params.N[0, 0]),
                                        int(params.M[0, 0]), float(sigma_r), int(gauss),
                                        _p(uy), _p(ux), uy.size, _p(ys), _p(xs), ys.size,
                                        _p(out), _p(num), _p(den))
    if points is None:
        out, num, den = out.reshape(H, W), num.reshape(H, W), den.reshape(H, W)
    if return_parts:
        return out, num, den, nfb
    return out


def nlm_shiftable(f, sigma_s: float, sigma_r: float, params: Params, patch_mask: int, *,
                  spatial: str = "box", return_parts=False):
    """The O(1) shiftable form of the same sums: one pair of modulated
    planes per multi-index of the product expansion (every multi-index,
    no folding)."""
    assert params.T.size == 1, "non-local means takes one (N, M)"
    f = _f64(f)
    H, W = f.shape
    uy, ux = patch_offsets(patch_mask)
    g = spatial_taps(sigma_s, params.R, spatial)
    out, num, den = np.empty_like(f), np.empty_like(f), np.empty_like(f)
    nfb = _load().orc_nlm_shiftable(_p(f), H, W, _p(g), params.R, int(params.N[0, 0]),
                                    int(params.M[0, 0]), float(sigma_r), _p(uy), _p(ux), uy.size,
                                    _p(out), _p(num), _p(den))
    if return_parts:
        return out, num, den, nfb
    return out


def _blocks(p: Params, H: int, W: int):
    ty, tx = p.T.shape
    for a in range(ty):
        for b in range(tx):
            y0, x0 = a * p.tile_h, b * p.tile_w
            yield a, b, y0, min(H, y0 + p.tile_h), x0, min(W, x0 + p.tile_w)


# ---------------------------------------------------------------- recursive filter

def yvv_coeffs(sigma: float) -> np.ndarray:
    """[B, b1/b0, b2/b0, b3/b0] of the Young-van Vliet recursion."""
    c = np.empty(4)
    _load().orc_yvv_coeffs(float(sigma), _p(c))
    return c


def yvv_margin(sigma: float) -> int:
    return _load().orc_yvv_margin(float(sigma))


def yvv_2d(img, sigma: float, margin: int = -1) -> np.ndarray:
    """Rows, then columns, of the recursion on the zero-extended image."""
    img = _f64(img)
    out = np.empty_like(img)
    _load().orc_yvv_2d(_p(img), _p(out), img.shape[0], img.shape[1], float(sigma), int(margin))
    return out


def yvv_impulse(sigma: float, half: int) -> np.ndarray:
    """h[d + half], d = -half..half."""
    h = np.empty(2 * half + 1)
    _load().orc_yvv_impulse(float(sigma), int(half), _p(h))
    return h


# ---------------------------------------------------------------- filters

def shiftable(f, sigma_s: float, sigma_r: float, params: Params, *, return_parts=False,
              spatial: str = "fir"):
    """SHIFTABLE-BF (Sec. 1.2) with phi_eps per T-tile.  Returns out (and
    num, den, number of guarded pixels when return_parts).  ``spatial``
    "yvv" filters the planes with the Young-van Vliet recursion instead of
    the truncated Gaussian (single kernel only); "box" with the constant
    filter of radius params.R (Sec. 4)."""
    f = _f64(f)
    H, W = f.shape
    if spatial == "yvv":
        assert params.T.size == 1, "the recursive mode takes one (N, M)"
        out, num, den = np.empty_like(f), np.empty_like(f), np.empty_like(f)
        nfb = _load().orc_shiftable_yvv(_p(f), H, W, float(sigma_s), int(params.N[0, 0]),
                                        int(params.M[0, 0]), float(sigma_r),
                                        _p(out), _p(num), _p(den))
        if return_parts:
            return out, num, den, nfb
        return out
    g = spatial_taps(sigma_s, params.R, spatial)
    out = np.empty_like(f)
    num = np.empty_like(f)
    den = np.empty_like(f)
    nfb = 0
    lib = _load()
    for a, b, y0, y1, x0, x1 in _blocks(params, H, W):
        nfb += lib.orc_shiftable_block(_p(f), H, W, _p(g), params.R,
                                       int(params.N[a, b]), int(params.M[a, b]),
                                       float(sigma_r), y0, y1, x0, x1,
                                       _p(out), _p(num), _p(den))
    if return_parts:
        return out, num, den, nfb
    return out


def _tile_of(params: Params, ys, xs):
    return ys // params.tile_h, xs // params.tile_w


def direct(f, sigma_s: float, sigma_r: float, params: Params | None = None, *,
           points=None, gauss: bool = False, return_parts=False, spatial: str = "fir"):
    """Direct sum of eq. (BF) at the given points (all pixels if None), with
    the range kernel phi_eps of each point's T-tile, or the Gaussian itself
    when ``gauss``.  Returns values in the order of ``points`` (or an image).
    ``spatial`` "yvv" weighs neighbours by the product of the recursion's
    one-dimensional impulse responses over the whole image instead of the
    truncated Gaussian; "box" weighs the (2 sigma_s + 1)^2 square equally."""
    f = _f64(f)
    H, W = f.shape
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = np.asarray(points[0]), np.asarray(points[1])
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    if spatial == "yvv":
        R = max(H, W)
        g = yvv_impulse(sigma_s, R)
    elif spatial in ("fir", "box"):
        if params is not None:
            R = params.R
        else:
            R = box_radius(sigma_s) if spatial == "box" else radius(sigma_s)
        g = spatial_taps(sigma_s, R, spatial)
    else:
        raise ValueError(spatial)
    if gauss:
        Ns = np.ones(ys.size, np.int32)
        Ms = np.zeros(ys.size, np.int32)
    else:
        a, b = _tile_of(params, ys, xs)
        Ns = np.ascontiguousarray(params.N[a, b], dtype=np.int32)
        Ms = np.ascontiguousarray(params.M[a, b], dtype=np.int32)
        # group by N so that the weights are rebuilt rarely
        order_ = np.argsort(Ns, kind="stable")
        inv = np.empty_like(order_)
        inv[order_] = np.arange(order_.size)
        ys, xs, Ns, Ms = (np.ascontiguousarray(v[order_]) for v in (ys, xs, Ns, Ms))
    out = np.empty(ys.size)
    num = np.empty(ys.size)
    den = np.empty(ys.size)
    nfb = _load().orc_direct_points(_p(f), H, W, _p(g), R, _p(Ns), _p(Ms), float(sigma_r),
                                    int(gauss), _p(ys), _p(xs), ys.size,
                                    _p(out), _p(num), _p(den))
    if not gauss:
        out, num, den = out[inv], num[inv], den[inv]
    if points is None:
        out, num, den = out.reshape(H, W), num.reshape(H, W), den.reshape(H, W)
    if return_parts:
        return out, num, den, nfb
    return out


def grad_shiftable(f, u, sigma_s: float, sigma_r: float, params: Params, *,
                   spatial: str = "fir"):
    """d/df of L = sum u * out, T, N, M held fixed (shiftable form)."""
    f = _f64(f)
    u = _f64(u)
    H, W = f.shape
    out, num, den, _ = shiftable(f, sigma_s, sigma_r, params, return_parts=True,
                                 spatial=spatial)
    g = spatial_taps(sigma_s, params.R, spatial)
    guarded = ~(den > 1e-6 * _mass(g, params.R, H, W))
    a = np.where(guarded, 0.0, u / np.where(guarded, 1.0, den))
    b = -a * out
    grad = np.where(guarded, u, 0.0)
    grad = np.ascontiguousarray(grad)
    lib = _load()
    for ta, tb, y0, y1, x0, x1 in _blocks(params, H, W):
        lib.orc_grad_shiftable_block(_p(f), H, W, _p(g), params.R,
                                     int(params.N[ta, tb]), int(params.M[ta, tb]),
                                     float(sigma_r), y0, y1, x0, x1,
                                     _p(np.ascontiguousarray(a)), _p(np.ascontiguousarray(b)),
                                     _p(grad))
    return grad


def grad_direct(f, u, sigma_s: float, sigma_r: float, params: Params, points=None, *,
                spatial: str = "fir"):
    """Same gradient from the direct form (single kernel only)."""
    assert params.T.size == 1, "direct gradient takes one (N, M)"
    f = _f64(f)
    u = _f64(u)
    H, W = f.shape
    out, num, den, _ = direct(f, sigma_s, sigma_r, params, return_parts=True, spatial=spatial)
    g = spatial_taps(sigma_s, params.R, spatial)
    guarded = ~(den > 1e-6 * _mass(g, params.R, H, W))
    a = np.ascontiguousarray(np.where(guarded, 0.0, u / np.where(guarded, 1.0, den)))
    b = np.ascontiguousarray(-a * out)
    if points is None:
        yy, xx = np.mgrid[0:H, 0:W]
        ys, xs = yy.ravel(), xx.ravel()
    else:
        ys, xs = np.asarray(points[0]), np.asarray(points[1])
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    res = np.empty(ys.size)
    _load().orc_grad_direct_points(_p(f), H, W, _p(g), params.R, int(params.N[0, 0]),
                                   int(params.M[0, 0]), float(sigma_r), _p(a), _p(b),
                                   _p(ys), _p(xs), ys.size, _p(res))
    res = res + np.where(guarded, u, 0.0).ravel()[ys * W + xs]
    if points is None:
        return res.reshape(H, W)
    return res


def _mass(g, R, H, W):
    """(g * 1_Omega) at every pixel (separable clipped sums)."""
    def line(n):
        m = np.empty(n)
        for i in range(n):
            lo, hi = max(0, i - R), min(n - 1, i + R)
            m[i] = g[lo - i + R: hi - i + R + 1].sum()
        return m
    return np.outer(line(H), line(W))
