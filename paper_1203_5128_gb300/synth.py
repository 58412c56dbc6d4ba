"""Seeded synthetic images standing in for the paper's test images.

The paper's Lena, Barbara and Checker images are not available (and the
Checker square size is not stated), so every workload uses one of two
seeded generators (numpy PCG64).  This module holds no part of the
filter's arithmetic; it is the one module that both the CUDA path's tests
and the oracle's tests import.

G8  -- 8-bit range [0, 255] (piecewise-constant, edges like Checker/Lena):
       background 0; max(8, H*W/4096) axis-aligned rectangles with uniform
       random corners and uniform [0, 255] intensity, painted in order; plus
       the ramp 32 (x/(W-1) + y/(H-1) - 1); plus N(0, 10^2) noise; clipped
       to [0, 255], not quantised.
G16 -- 16-bit range [0, 65535] (smooth field with step edges):
       4 octaves of bilinear value noise (lattice (4*2^o+1)^2, amplitude
       0.5^o) rescaled to [8000, 56000]; plus 8 random half-plane steps of
       +-U(4000, 16000); plus N(0, 300^2) noise; clipped to [0, 65535].
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def g8(H: int, W: int, seed: int = 0) -> np.ndarray:
    """8-bit-range test image, float32 [H, W]."""
    rng = _rng(seed)
    img = np.zeros((H, W), np.float32)
    nrect = max(8, (H * W) // 4096)
    ys = rng.integers(0, H, size=(nrect, 2))
    xs = rng.integers(0, W, size=(nrect, 2))
    val = rng.uniform(0.0, 255.0, size=nrect).astype(np.float32)
    ys.sort(axis=1)
    xs.sort(axis=1)
    for k in range(nrect):
        img[ys[k, 0]:ys[k, 1] + 1, xs[k, 0]:xs[k, 1] + 1] = val[k]
    x = np.arange(W, dtype=np.float64) / max(W - 1, 1)
    y = np.arange(H, dtype=np.float64) / max(H - 1, 1)
    ramp = 32.0 * (x[None, :] + y[:, None] - 1.0)
    noise = rng.normal(0.0, 10.0, size=(H, W))
    out = img.astype(np.float64) + ramp + noise
    return np.clip(out, 0.0, 255.0).astype(np.float32)


def _value_noise(rng: np.random.Generator, H: int, W: int, L: int) -> np.ndarray:
    lat = rng.uniform(0.0, 1.0, size=(L, L))
    v = np.arange(H, dtype=np.float64) * (L - 1) / max(H - 1, 1)
    u = np.arange(W, dtype=np.float64) * (L - 1) / max(W - 1, 1)
    i0 = np.minimum(np.floor(v).astype(np.int64), L - 2)
    j0 = np.minimum(np.floor(u).astype(np.int64), L - 2)
    fy = (v - i0)[:, None]
    fx = (u - j0)[None, :]
    a = lat[i0][:, j0]
    b = lat[i0][:, j0 + 1]
    c = lat[i0 + 1][:, j0]
    d = lat[i0 + 1][:, j0 + 1]
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy


def g16(H: int, W: int, seed: int = 2) -> np.ndarray:
    """16-bit-range test image, float32 [H, W]."""
    rng = _rng(seed)
    field = np.zeros((H, W))
    for o in range(4):
        field += 0.5 ** o * _value_noise(rng, H, W, 4 * 2 ** o + 1)
    lo, hi = field.min(), field.max()
    field = 8000.0 + (field - lo) * (48000.0 / max(hi - lo, 1e-12))
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(8):
        py, px = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        amp = rng.uniform(4000.0, 16000.0) * (1.0 if rng.uniform() < 0.5 else -1.0)
        side = (xx - px) * np.cos(ang) + (yy - py) * np.sin(ang) > 0.0
        field = field + amp * side
    field = field + rng.normal(0.0, 300.0, size=(H, W))
    return np.clip(field, 0.0, 65535.0).astype(np.float32)


def batch_specs(n: int = 64, seed: int = 3):
    """Per-image (H, W, sigma_s, sigma_r) of the batched workload: sides
    uniform in [128, 2048] (non-square), sigma_s in [2, 16], sigma_r in
    [10, 60], all drawn from the seed."""
    rng = _rng(seed)
    H = rng.integers(128, 2049, size=n)
    W = rng.integers(128, 2049, size=n)
    ss = rng.uniform(2.0, 16.0, size=n)
    sr = rng.uniform(10.0, 60.0, size=n)
    return [(int(H[i]), int(W[i]), float(ss[i]), float(sr[i])) for i in range(n)]


def weights_normal(shape, seed: int = 4) -> np.ndarray:
    """The seeded N(0, 1) weight image w of the loss L = sum(w * out)."""
    return _rng(seed).normal(0.0, 1.0, size=shape).astype(np.float32)
