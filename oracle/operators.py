"""Forward operators A and their adjoints (FP64 oracle).

* Gaussian blur (Section 3.1): a (2r+1)-tap sampled Gaussian, normalised to unit sum,
  applied separably along both image axes with half-sample symmetric extension
  ("... b a | a b ...").  ``blur`` gathers; ``blur_adjoint`` is the literal transpose,
  built by scattering each output's taps back onto the input.
* Parallel-beam projector (Section 3.3, the discrete Radon transform): a ray-driven
  projector in Joseph's discretisation.  ``joseph_forward`` sums linear interpolations
  along each ray; ``joseph_adjoint`` scatters the same weights back (literal transpose).

Geometry of the projector: an N x N image with pixel size s spans [-Ns/2, Ns/2]^2;
pixel (i, j) has centre (x_j, y_i) = ((j - (N-1)/2) s, (i - (N-1)/2) s).  Angle
theta_a = a pi / n_angles, detector direction (cos, sin), ray direction (-sin, cos);
bin b sits at t_b = (b - (n_det-1)/2) s_det and its ray is {x cos + y sin = t_b}.
When |cos| >= |sin| the ray is walked row by row (y = y_i, interpolating along x);
otherwise column by column.  Each sample has weight s / max(|cos|, |sin|); pixels
outside the image count as zero.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ---------------------------------------------------------------- blur
def gaussian_weights(sigma: float, radius: int = 4) -> np.ndarray:
    """w_i = exp(-i^2 / (2 sigma^2)), i = -radius..radius, normalised to sum 1."""
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-(i * i) / (2.0 * sigma * sigma))
    return w / w.sum()


def reflect_index(j, n):
    """Half-sample symmetric extension of index j into [0, n)."""
    j = np.mod(j, 2 * n)
    return np.where(j >= n, 2 * n - 1 - j, j)


def _blur_axis(u, w, axis):
    r = (len(w) - 1) // 2
    n = u.shape[axis]
    out = np.zeros_like(u)
    idx = np.arange(n)
    for k, wk in enumerate(w):
        src = reflect_index(idx + (k - r), n)
        out += wk * np.take(u, src, axis=axis)
    return out


def _blur_axis_adjoint(y, w, axis):
    r = (len(w) - 1) // 2
    n = y.shape[axis]
    out = np.zeros_like(y)
    idx = np.arange(n)
    for k, wk in enumerate(w):
        dst = reflect_index(idx + (k - r), n)
        contrib = wk * y
        if axis == 0:
            np.add.at(out, dst, contrib)
        else:
            np.add.at(out.T, dst, contrib.T)
    return out


def blur(u: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A u: separable blur with taps ``w`` along x then y, symmetric boundary."""
    u = np.asarray(u, dtype=np.float64)
    return _blur_axis(_blur_axis(u, w, 1), w, 0)


def blur_adjoint(y: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A^T y by scattering every tap of every output sample back to its source."""
    y = np.asarray(y, dtype=np.float64)
    return _blur_axis_adjoint(_blur_axis_adjoint(y, w, 0), w, 1)


# ---------------------------------------------------------------- projector
@dataclass(frozen=True)
class ParallelBeam:
    """Parallel-beam geometry (see the module docstring)."""
    N: int
    n_angles: int
    n_det: int
    pixel_size: float
    det_spacing: float

    @staticmethod
    def unit_square(N, n_angles, n_det):
        """Image of unit side length (s = 1/N), bins of pixel width."""
        return ParallelBeam(N, n_angles, n_det, 1.0 / N, 1.0 / N)

    def angles(self):
        return np.arange(self.n_angles, dtype=np.float64) * math.pi / self.n_angles

    def bins(self):
        return (np.arange(self.n_det, dtype=np.float64) - (self.n_det - 1) / 2.0) * self.det_spacing


def _ray_samples(geom: ParallelBeam, a: int):
    """For angle index a: (row_major, idx_line, i0, f, weight) over (lines, bins).

    row_major is True when the ray is walked over rows.  For line l (a row index if
    row_major else a column index) and bin b, the ray crosses the line at fractional
    pixel coordinate c = i0 + f along the line, i0 = floor(c).
    """
    N, s = geom.N, geom.pixel_size
    th = a * math.pi / geom.n_angles
    c, sn = math.cos(th), math.sin(th)
    t = geom.bins()[None, :]
    lines = np.arange(N, dtype=np.float64)[:, None]
    coord = (lines - (N - 1) / 2.0) * s
    if abs(c) >= abs(sn):
        pos = (t - coord * sn) / c          # x where the ray meets row y_i
        weight = s / abs(c)
        row_major = True
    else:
        pos = (t - coord * c) / sn          # y where the ray meets column x_j
        weight = s / abs(sn)
        row_major = False
    frac_idx = pos / s + (N - 1) / 2.0
    i0 = np.floor(frac_idx)
    f = frac_idx - i0
    return row_major, i0.astype(np.int64), f, weight


def joseph_forward(u: np.ndarray, geom: ParallelBeam) -> np.ndarray:
    """Sinogram (n_angles, n_det) of line integrals through ``u`` (Joseph)."""
    u = np.asarray(u, dtype=np.float64)
    N = geom.N
    sino = np.zeros((geom.n_angles, geom.n_det), dtype=np.float64)
    lines = np.arange(N)[:, None]
    for a in range(geom.n_angles):
        row_major, i0, f, weight = _ray_samples(geom, a)
        acc = np.zeros(i0.shape)
        for off, wgt in ((0, 1.0 - f), (1, f)):
            k = i0 + off
            ok = (k >= 0) & (k < N)
            kc = np.clip(k, 0, N - 1)
            vals = u[lines, kc] if row_major else u[kc, lines]
            acc += np.where(ok, wgt * vals, 0.0)
        sino[a] = weight * acc.sum(axis=0)
    return sino


def joseph_adjoint(y: np.ndarray, geom: ParallelBeam) -> np.ndarray:
    """Back-projection A^T y: scatter of the forward weights."""
    y = np.asarray(y, dtype=np.float64)
    N = geom.N
    img = np.zeros((N, N), dtype=np.float64)
    lines = np.broadcast_to(np.arange(N)[:, None], (N, geom.n_det))
    for a in range(geom.n_angles):
        row_major, i0, f, weight = _ray_samples(geom, a)
        ya = np.broadcast_to(y[a][None, :], i0.shape)
        for off, wgt in ((0, 1.0 - f), (1, f)):
            k = i0 + off
            ok = (k >= 0) & (k < N)
            val = (weight * wgt * ya)[ok]
            if row_major:
                np.add.at(img, (lines[ok], k[ok]), val)
            else:
                np.add.at(img, (k[ok], lines[ok]), val)
    return img


# ---------------------------------------------------------------- operator bundles
@dataclass
class LinearOp:
    """A linear map with its adjoint, for the solvers."""
    forward: callable
    adjoint: callable
    name: str = "op"


def identity_op():
    return LinearOp(lambda x: np.array(x, dtype=np.float64),
                    lambda y: np.array(y, dtype=np.float64), "identity")


def blur_op(sigma: float, radius: int = 4):
    w = gaussian_weights(sigma, radius)
    return LinearOp(lambda x: blur(x, w), lambda y: blur_adjoint(y, w), "blur")


def ct_op(geom: ParallelBeam):
    return LinearOp(lambda x: joseph_forward(x, geom), lambda y: joseph_adjoint(y, geom), "ct")
