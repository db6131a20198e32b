"""Seeded phantoms and noise draws.

Every generator takes an explicit integer seed and uses numpy's PCG64, so the same
call gives the same array on every machine.  Shapes are painted in draw order; a
later shape overwrites an earlier one where they overlap.  All outputs are float64
arrays; callers that feed the CUDA path cast them to float32 and give the oracle the
float64 copy of those float32 values, so both sides see identical inputs.
"""

from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """numpy PCG64 generator for an integer seed."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _pixel_grid(n_rows: int, n_cols: int):
    yy = np.arange(n_rows, dtype=np.float64)[:, None] + 0.5
    xx = np.arange(n_cols, dtype=np.float64)[None, :] + 0.5
    return yy, xx


def shapes_phantom_2d(H: int, W: int, n_shapes: int, seed: int,
                      intensity=(0.0, 1.0), kinds=("rect", "ellipse")) -> np.ndarray:
    """Random axis-aligned rectangles and rotated ellipses on a zero background.

    Centres are uniform over [0.15, 0.85] of each side, semi-axes uniform in
    [0.03, 0.3] of the side, ellipse angles uniform in [0, pi), intensities uniform in
    ``intensity``; the kind of each shape alternates through ``kinds``.
    """
    g = rng(seed)
    img = np.zeros((H, W), dtype=np.float64)
    yy, xx = _pixel_grid(H, W)
    for s in range(n_shapes):
        kind = kinds[s % len(kinds)]
        cy = g.uniform(0.15, 0.85) * H
        cx = g.uniform(0.15, 0.85) * W
        ay = g.uniform(0.03, 0.3) * H
        ax = g.uniform(0.03, 0.3) * W
        ang = g.uniform(0.0, math.pi)
        val = g.uniform(*intensity)
        if kind == "rect":
            mask = (np.abs(yy - cy) <= ay) & (np.abs(xx - cx) <= ax)
        else:
            c, s_ = math.cos(ang), math.sin(ang)
            dy, dx = yy - cy, xx - cx
            e1 = (dx * c + dy * s_) / ax
            e2 = (-dx * s_ + dy * c) / ay
            mask = e1 * e1 + e2 * e2 <= 1.0
        img[mask] = val
    return img


def ellipses_phantom_2d(N: int, n_ellipses: int, seed: int,
                        intensity=(0.0, 1.0), W: int | None = None) -> np.ndarray:
    """N x W (default square) image of rotated ellipses, painter's order."""
    return shapes_phantom_2d(N, W if W is not None else N, n_ellipses, seed,
                             intensity=intensity, kinds=("ellipse",))


def ellipsoids_phantom_3d(N: int, n_ellipsoids: int, seed: int,
                          intensity=(0.0, 1.0), dtype=np.float32) -> np.ndarray:
    """N^3 volume of axis-aligned ellipsoids, painter's order.

    Each ellipsoid is evaluated only over its bounding box, so a 512^3 volume takes
    seconds.  Stored in ``dtype`` (float32 by default, to keep 512^3 at 0.5 GB).
    """
    g = rng(seed)
    vol = np.zeros((N, N, N), dtype=dtype)
    for _ in range(n_ellipsoids):
        c = g.uniform(0.15, 0.85, size=3) * N
        a = g.uniform(0.03, 0.3, size=3) * N
        val = g.uniform(*intensity)
        lo = np.maximum(np.floor(c - a).astype(int), 0)
        hi = np.minimum(np.ceil(c + a).astype(int) + 1, N)
        z = (np.arange(lo[0], hi[0]) + 0.5 - c[0])[:, None, None] / a[0]
        y = (np.arange(lo[1], hi[1]) + 0.5 - c[1])[None, :, None] / a[1]
        x = (np.arange(lo[2], hi[2]) + 0.5 - c[2])[None, None, :] / a[2]
        mask = z * z + y * y + x * x <= 1.0
        sub = vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        sub[mask] = val
    return vol


def gaussian_noise(shape, sigma: float, seed: int, dtype=np.float64) -> np.ndarray:
    """i.i.d. N(0, sigma^2) samples."""
    g = rng(seed)
    return (g.standard_normal(size=shape, dtype=np.float64) * sigma).astype(dtype, copy=False)


def poisson_counts(expected: np.ndarray, seed: int) -> np.ndarray:
    """Independent Poisson draws with the given (non-negative) means."""
    g = rng(seed)
    return g.poisson(np.asarray(expected, dtype=np.float64)).astype(np.float64)


def batch_problem_specs(n: int, seed: int, lo: int = 64, hi: int = 1024):
    """Per-problem parameters of the uneven batch workload.

    Heights and widths are drawn independently and log-uniformly in [lo, hi]
    (round(lo * (hi/lo)^U)); problems alternate between denoising (even index) and
    9x9 Gaussian deblurring (odd index); alpha ~ U[0.01, 0.2], p ~ U[0.05, 0.5],
    blur sigma ~ U[1, 3]; the Philox seed of problem i is i.
    """
    g = rng(seed)
    ratio = hi / lo
    specs = []
    for i in range(n):
        H = int(round(lo * ratio ** g.uniform()))
        W = int(round(lo * ratio ** g.uniform()))
        alpha = g.uniform(0.01, 0.2)
        p = g.uniform(0.05, 0.5)
        blur_sigma = g.uniform(1.0, 3.0)
        specs.append(dict(index=i, H=H, W=W, kind="denoise" if i % 2 == 0 else "deblur",
                          alpha=alpha, p=p, blur_sigma=blur_sigma, seed=i))
    return specs
