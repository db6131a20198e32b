"""Pins of the oracle's blur and parallel-beam projector."""

import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import operators as op
from oracle.power import power_method


def _rng(seed=0):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("shape,sigma", [((17, 23), 2.0), ((3, 5), 1.0), ((64, 40), 2.7), ((1, 9), 1.5)])
def test_blur_matches_scipy_reflect(shape, sigma):
    """Half-sample symmetric separable blur equals scipy's correlate1d(mode='reflect')."""
    u = _rng(0).standard_normal(shape)
    w = op.gaussian_weights(sigma, 4)
    ref = ndi.correlate1d(ndi.correlate1d(u, w, axis=1, mode="reflect"), w, axis=0, mode="reflect")
    np.testing.assert_allclose(op.blur(u, w), ref, atol=1e-14)


def test_gaussian_weights():
    w = op.gaussian_weights(2.0, 4)
    assert len(w) == 9 and abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w / w[4], [math.exp(-i * i / 8.0) for i in range(-4, 5)], rtol=1e-15)


@pytest.mark.parametrize("shape", [(17, 23), (5, 3), (32, 32)])
def test_blur_dot_test_and_symmetry(shape):
    """<A u, y> = <u, A^T y> with A^T the literal scatter transpose; A = A^T."""
    g = _rng(1)
    u, y = g.standard_normal(shape), g.standard_normal(shape)
    w = op.gaussian_weights(1.7, 4)
    lhs = float(np.sum(op.blur(u, w) * y))
    rhs = float(np.sum(u * op.blur_adjoint(y, w)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    np.testing.assert_allclose(op.blur_adjoint(y, w), op.blur(y, w), atol=1e-14)


def test_blur_constant_and_norm():
    """A const = const (sum w = 1) and ||A|| = 1 (A is symmetric and doubly stochastic)."""
    w = op.gaussian_weights(2.0, 4)
    c = np.full((9, 7), 0.25)
    np.testing.assert_allclose(op.blur(c, w), c, atol=1e-15)
    shape = (8, 6)
    n = 48
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = op.blur(e.reshape(shape), w).ravel()
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    ev = np.linalg.eigvalsh(M)
    # symmetric with non-negative entries and unit row sums: spectral radius exactly 1
    assert abs(ev.max() - 1.0) < 1e-12 and np.abs(ev).max() < 1.0 + 1e-12
    lam = power_method(lambda x: op.blur(op.blur(x, w), w), shape, n_iter=2000)
    assert abs(lam - 1.0) < 1e-6


@pytest.mark.parametrize("N,na,nd", [(8, 12, 13), (16, 30, 23), (9, 7, 11)])
def test_joseph_dot_test(N, na, nd):
    geom = op.ParallelBeam.unit_square(N, na, nd)
    g = _rng(2)
    u = g.standard_normal((N, N))
    y = g.standard_normal((na, nd))
    lhs = float(np.sum(op.joseph_forward(u, geom) * y))
    rhs = float(np.sum(u * op.joseph_adjoint(y, geom)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_joseph_axis_aligned_hand_values():
    """4x4 image, 5 bins, 4 angles.  At theta = 0 bin b's ray is the vertical line
    halfway between pixel columns b-1 and b, so the sinogram is s * sum_i (u[i,b-1] +
    u[i,b]) / 2; at theta = pi/2 the same holds with rows and columns swapped."""
    N, s = 4, 0.25
    geom = op.ParallelBeam.unit_square(N, 4, 5)
    u = _rng(3).standard_normal((N, N))
    sino = op.joseph_forward(u, geom)
    pad = np.zeros((N + 2, N + 2))
    pad[1:-1, 1:-1] = u
    for b in range(5):
        col_pair = 0.5 * (pad[1:-1, b] + pad[1:-1, b + 1])
        row_pair = 0.5 * (pad[b, 1:-1] + pad[b + 1, 1:-1])
        assert sino[0, b] == pytest.approx(s * col_pair.sum(), abs=1e-14)
        assert sino[2, b] == pytest.approx(s * row_pair.sum(), abs=1e-12)


def test_joseph_disc_line_integrals():
    """Sanity (not exact for Joseph): a disc of radius r has line integrals 2 sqrt(r^2 - t^2)."""
    N = 128
    geom = op.ParallelBeam.unit_square(N, 8, 183)
    yy, xx = np.mgrid[0:N, 0:N]
    x = (xx - (N - 1) / 2) / N
    y = (yy - (N - 1) / 2) / N
    r = 0.3
    disc = (x * x + y * y <= r * r).astype(float)
    sino = op.joseph_forward(disc, geom)
    t = geom.bins()
    expect = 2 * np.sqrt(np.maximum(r * r - t * t, 0))
    err = np.abs(sino - expect[None, :])
    assert err[:, np.abs(t) < 0.25].max() < 0.02      # away from the tangent rays
    assert err.mean() < 0.005
    # mass: sum_b sino[a, b] * s_det ~ s^2 sum u
    mass = sino.sum(axis=1) * geom.det_spacing
    np.testing.assert_allclose(mass, disc.sum() / N ** 2, rtol=1e-2)


def test_joseph_norm_by_power_method():
    geom = op.ParallelBeam.unit_square(16, 24, 23)
    lam = power_method(lambda x: op.joseph_adjoint(op.joseph_forward(x, geom), geom), (16, 16), n_iter=300)
    # dense check of the same quantity
    n = 256
    M = np.zeros((24 * 23, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = op.joseph_forward(e.reshape(16, 16), geom).ravel()
    assert abs(lam - np.linalg.norm(M, 2) ** 2) < 1e-8 * lam
