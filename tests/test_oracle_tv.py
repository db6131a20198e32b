"""Pins of the oracle's D, div, TV and TV prox against facts fixed by the mathematics.

Each check uses a route that does not go through the function under test: numpy's
diff, dense eigenvalues, closed forms, a box-constrained least-squares library solve,
and weak duality evaluated by explicit loops.
"""

import math

import numpy as np
import pytest
from scipy.optimize import lsq_linear

from oracle import tv


def _rng(seed=0):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("shape", [(7, 5), (1, 9), (9, 1), (16, 16), (4, 5, 6), (1, 3, 7), (33, 17)])
def test_adjoint_identity(shape):
    """<D u, p> = -<u, div p> (div = -D^T, Section 2.1) to 1e-12 relative."""
    g = _rng(1)
    u = g.standard_normal(shape)
    p = g.standard_normal((len(shape),) + shape)
    lhs = float(np.sum(tv.grad(u) * p))
    rhs = -float(np.sum(u * tv.div(p)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("shape", [(6, 8), (3, 4, 5)])
def test_grad_matches_numpy_diff(shape):
    """Forward differences with a zero last difference (Neumann) equal numpy's diff."""
    u = _rng(2).standard_normal(shape)
    g = tv.grad(u)
    for a in range(len(shape)):
        ref = np.diff(u, axis=a)
        pad = [(0, 0)] * len(shape)
        pad[a] = (0, 1)
        np.testing.assert_array_equal(g[a], np.pad(ref, pad))


@pytest.mark.parametrize("shape", [(5, 7), (8, 8), (3, 4, 5)])
def test_norm_D_closed_form(shape):
    """||D||^2 = sum_a 4 sin^2(pi (n_a - 1) / (2 n_a)) (the DCT-II diagonalises D^T D).

    The dense matrix D^T D is assembled column by column from the oracle's grad/div
    and its largest eigenvalue compared with the closed form; the value is <= 4 d.
    """
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = -tv.div(tv.grad(e.reshape(shape))).ravel()
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    lam_max = np.linalg.eigvalsh(M).max()
    closed = sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in shape)
    assert abs(lam_max - closed) < 1e-10
    assert lam_max <= 4.0 * len(shape)


def test_power_method_norm_D():
    from oracle.power import power_method
    shape = (6, 9)
    lam = power_method(lambda x: -tv.div(tv.grad(x)), shape, n_iter=3000)
    closed = sum(4.0 * math.sin(math.pi * (m - 1) / (2.0 * m)) ** 2 for m in shape)
    assert abs(lam - closed) < 1e-8


def test_tv_closed_forms():
    """TV of a vertical step of height 1 is H; TV of u = i + j is known in closed form."""
    H, W = 6, 9
    step = np.zeros((H, W))
    step[:, 4:] = 1.0
    assert tv.tv(step) == pytest.approx(H, abs=1e-13)
    ramp = np.add.outer(np.arange(H), np.arange(W)).astype(float)
    expect = (H - 1) * (W - 1) * math.sqrt(2.0) + (H - 1) + (W - 1)
    assert tv.tv(ramp) == pytest.approx(expect, rel=1e-14)
    cube = np.zeros((3, 4, 5))
    cube[:, :, 2:] = 2.0
    assert tv.tv(cube) == pytest.approx(2.0 * 3 * 4, rel=1e-14)


def test_prox_lambda_zero_is_identity():
    z = _rng(3).standard_normal((9, 11))
    u, _ = tv.fgp_prox(z, 0.0, 50)
    np.testing.assert_array_equal(u, z)


def test_prox_constant_image_unchanged():
    z = np.full((7, 5), 0.37)
    u, p = tv.fgp_prox(z, 0.8, 40)
    np.testing.assert_allclose(u, z, atol=1e-15)
    assert np.all(p == 0.0)


@pytest.mark.parametrize("z1,z2,lam", [(0.0, 1.0, 0.1), (0.3, 0.2, 0.2), (2.0, -1.0, 0.4)])
@pytest.mark.parametrize("orient", ["row", "col"])
def test_prox_two_pixel_closed_form(z1, z2, lam, orient):
    """Two pixels: if |z1 - z2| <= 2 lam both become the mean, else each moves lam
    toward the other (minimiser of 1/2 (u1-z1)^2 + 1/2 (u2-z2)^2 + lam |u2 - u1|)."""
    z = np.array([[z1, z2]]) if orient == "row" else np.array([[z1], [z2]])
    u, _ = tv.fgp_prox(z, lam, 3000)
    if abs(z1 - z2) <= 2 * lam:
        expect = [(z1 + z2) / 2] * 2
    else:
        sgn = math.copysign(1.0, z2 - z1)
        expect = [z1 + sgn * lam, z2 - sgn * lam]
    np.testing.assert_allclose(u.ravel(), expect, atol=1e-10)


def test_prox_preserves_mean():
    """sum(div p) = 0, so sum u = sum z for every iterate (no constraint)."""
    z = _rng(4).standard_normal((13, 10))
    for n in (1, 5, 37):
        u, _ = tv.fgp_prox(z, 0.3, n)
        assert abs(u.sum() - z.sum()) < 1e-12 * z.size


def test_prox_huge_lambda_gives_mean():
    z = _rng(5).standard_normal((3, 4))
    u, _ = tv.fgp_prox(z, 50.0, 20000)
    np.testing.assert_allclose(u, np.full_like(z, z.mean()), atol=1e-8)


def _exact_1d_tv_prox(z, lam):
    """Exact prox of lam * sum |u_{i+1} - u_i| through its box-constrained dual,
    min_q 1/2 || z - lam M q ||^2 with -1 <= q <= 1 and (M q)_i = q_{i-1} - q_i,
    solved by bounded-variable least squares (scipy)."""
    n = len(z)
    M = np.zeros((n, n - 1))
    for i in range(n - 1):
        M[i, i] = -1.0
        M[i + 1, i] = 1.0
    res = lsq_linear(lam * M, z, bounds=(-1.0, 1.0), method="bvls", tol=1e-15, max_iter=10000)
    return z - lam * M @ res.x


@pytest.mark.parametrize("n,lam,seed", [(7, 0.3, 0), (12, 0.15, 1), (5, 1.0, 2)])
def test_prox_1d_matches_exact_solver(n, lam, seed):
    """A 1 x n (or n x 1) image has isotropic TV equal to 1D TV; compare with an exact
    box-QP solve of the 1D dual."""
    z = _rng(seed).standard_normal(n)
    exact = _exact_1d_tv_prox(z, lam)
    u_row, _ = tv.fgp_prox(z[None, :], lam, 20000)
    u_col, _ = tv.fgp_prox(z[:, None], lam, 20000)
    np.testing.assert_allclose(u_row.ravel(), exact, atol=1e-9)
    np.testing.assert_allclose(u_col.ravel(), exact, atol=1e-9)


def _primal_by_loops(u, z, lam):
    H, W = u.shape
    val = 0.0
    for i in range(H):
        for j in range(W):
            dy = u[i + 1, j] - u[i, j] if i + 1 < H else 0.0
            dx = u[i, j + 1] - u[i, j] if j + 1 < W else 0.0
            val += 0.5 * (u[i, j] - z[i, j]) ** 2 + lam * math.sqrt(dy * dy + dx * dx)
    return val


def _dual_by_loops(p, z, lam):
    """1/2||z||^2 - 1/2||z - lam D^T p||^2, D^T p assembled pixel by pixel."""
    H, W = z.shape
    DTp = np.zeros_like(z)
    for i in range(H):
        for j in range(W):
            if i + 1 < H:
                DTp[i + 1, j] += p[0, i, j]
                DTp[i, j] -= p[0, i, j]
            if j + 1 < W:
                DTp[i, j + 1] += p[1, i, j]
                DTp[i, j] -= p[1, i, j]
    w = z - lam * DTp
    return 0.5 * float(np.sum(z * z)) - 0.5 * float(np.sum(w * w)), z - lam * DTp


def test_prox_4x4_weak_duality_certificate():
    """For any |p_i| <= 1, D(p) <= P(u*) <= P(u).  With both evaluated by explicit
    loops, P(u) - D(p) < 1e-12 certifies ||u - u*||^2 <= 2e-12 (P is 1-strongly convex)."""
    z = _rng(6).standard_normal((4, 4))
    lam = 0.35
    u, p = tv.fgp_prox(z, lam, 20000)
    assert np.sqrt((p ** 2).sum(axis=0)).max() <= 1.0 + 1e-15
    d_val, u_from_p = _dual_by_loops(p, z, lam)
    np.testing.assert_allclose(u, u_from_p, atol=1e-14)
    gap = _primal_by_loops(u, z, lam) - d_val
    assert -1e-13 <= gap < 1e-12
    # second route: plain (non-accelerated) dual projected gradient
    u2, _ = tv.projgd_prox(z, lam, 200000)
    np.testing.assert_allclose(u2, u, atol=1e-9)


def test_rof_gap_nonnegative_and_vanishing():
    z = _rng(7).standard_normal((10, 12))
    lam = 0.2
    gaps = []
    p = None
    for _ in range(30):
        _, p = tv.fgp_prox(z, lam, 50, p)
        gaps.append(tv.rof_gap(z, lam, p))
    assert min(gaps) >= -1e-12
    assert gaps[-1] < 1e-9 * tv.rof_primal(z + lam * tv.div(p), z, lam)


def test_prox_nonneg_clips():
    z = _rng(8).standard_normal((6, 6))
    u, _ = tv.fgp_prox(z, 0.1, 200, nonneg=True)
    assert u.min() >= 0.0
    # with a non-negative z and tiny lambda the clip is inactive
    u2, _ = tv.fgp_prox(np.abs(z) + 1.0, 1e-3, 200, nonneg=True)
    u3, _ = tv.fgp_prox(np.abs(z) + 1.0, 1e-3, 200, nonneg=False)
    np.testing.assert_allclose(u2, u3, atol=1e-14)
