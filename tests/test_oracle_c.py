"""The oracle's C transcription (oracle/tvo.c) against the numpy oracle.

tvo.c restates the numpy oracle loop for loop so that full-size oracle runs (the
reference optimum of the 1024 x 1024 deblurring workload, the CPU baseline on every
host core) are affordable.  It is pinned to the numpy functions, which carry the
pins against the paper and the mathematics: equal to 1e-12 (in practice bit for bit
except for sums over the image, which OpenMP reduces in another order).
"""

import numpy as np
import pytest

from oracle import c, coin, operators, solvers, tv


def _z(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (13, 17), (4, 5, 6), (1, 3, 7), (6, 1, 1)])
def test_grad_div_tv(shape):
    u = _z(shape, 1)
    p = _z((len(shape),) + shape, 2)
    np.testing.assert_array_equal(c.grad(u), tv.grad(u))
    np.testing.assert_array_equal(c.div(p), tv.div(p))
    assert c.tv(u) == pytest.approx(tv.tv(u), rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("shape,lam,n,nonneg", [((13, 17), 0.2, 23, False), ((13, 17), 0.02, 5, True),
                                                ((1, 2), 0.25, 4, False), ((4, 5, 6), 0.15, 9, False),
                                                ((4, 5, 6), 0.3, 7, True), ((8, 8), 0.0, 5, False)])
def test_fgp_prox(shape, lam, n, nonneg):
    z = _z(shape, 3)
    p0 = tv.project_unit_ball(_z((len(shape),) + shape, 4))
    for warm in (None, p0):
        u1, p1 = tv.fgp_prox(z, lam, n, warm, nonneg)
        u2, p2 = c.fgp_prox(z, lam, n, warm, nonneg)
        np.testing.assert_allclose(u2, u1, rtol=0, atol=1e-12)
        np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,sigma,radius", [((16, 11), 1.5, 4), ((3, 40), 2.0, 4), ((9, 9), 1.0, 8),
                                                ((2, 2), 2.0, 4)])
def test_blur_and_adjoint(shape, sigma, radius):
    u = _z(shape, 5)
    w = operators.gaussian_weights(sigma, radius)
    np.testing.assert_allclose(c.blur(u, w), operators.blur(u, w), rtol=0, atol=1e-13)
    np.testing.assert_allclose(c.blur(u, w, adjoint=True), operators.blur_adjoint(u, w), rtol=0, atol=1e-13)


def _deblur(n=14, seed=6, alpha=0.03):
    g = np.random.default_rng(seed)
    truth = np.zeros((n, n + 3))
    truth[2:8, 3:11] = 1.0
    truth[7:12, 1:6] = 0.5
    w = operators.gaussian_weights(1.5)
    b = operators.blur(truth, w) + 0.01 * g.standard_normal(truth.shape)
    return b, w, alpha


def test_objective():
    b, w, alpha = _deblur()
    x = _z(b.shape, 7)
    prob = solvers.Problem(operators.blur_op(1.5), b, alpha, b.shape)
    assert c.objective(b, alpha, x, w) == pytest.approx(prob.objective(x), rel=1e-13)
    prob_i = solvers.Problem(operators.identity_op(), b, alpha, b.shape)
    assert c.objective(b, alpha, x) == pytest.approx(prob_i.objective(x), rel=1e-13)


@pytest.mark.parametrize("op", ["blur", "identity"])
@pytest.mark.parametrize("kind", ["pgd", "fista", "proxskip"])
def test_fb_solvers(op, kind):
    b, w, alpha = _deblur()
    A = operators.blur_op(1.5) if op == "blur" else operators.identity_op()
    prob = solvers.Problem(A, b, alpha, b.shape)
    gamma, K, N, p, seed = (1.0 if op == "blur" else 0.7), 18, 6, 0.35, 9
    if kind == "pgd":
        ref = solvers.pgd(prob, b, gamma, K, N)
    elif kind == "fista":
        ref = solvers.fista(prob, b, gamma, K, N)
    else:
        ref = solvers.proxskip(prob, b, gamma, p, seed, K, N)
    got = c.fb_solve(kind, b, alpha, gamma, K, N, w=w if op == "blur" else None, p=p,
                     coins=coin.schedule(seed, p, K) if kind == "proxskip" else None)
    np.testing.assert_allclose(got["x"], ref["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["dual"], ref["dual"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["objective"], ref["objective"], rtol=1e-12)
    assert got["prox_calls"] == ref["prox_calls"] and got["iters_run"] == K


def test_fb_solver_3d_identity_and_stop():
    """3D denoising (identity operator), and the stop at a relative-gap target."""
    b = _z((5, 6, 7), 10)
    prob = solvers.Problem(operators.identity_op(), b, 0.1, b.shape)
    ref = solvers.proxskip(prob, b, 1.0, 0.5, 3, 12, 5)
    got = c.fb_solve("proxskip", b, 0.1, 1.0, 12, 5, p=0.5, coins=coin.schedule(3, 0.5, 12))
    np.testing.assert_allclose(got["x"], ref["x"], rtol=0, atol=1e-12)
    f_star = min(ref["objective"]) * (1 - 1e-6)
    k_hit = next(k for k, F in enumerate(ref["objective"]) if (F - f_star) / f_star <= 1e-3)
    stop = c.fb_solve("proxskip", b, 0.1, 1.0, 12, 5, p=0.5, coins=coin.schedule(3, 0.5, 12),
                      f_star=f_star, target=1e-3)
    assert stop["iters_run"] == k_hit + 1


@pytest.mark.parametrize("N,na,nd,spacing", [(24, 37, 31, None), (17, 20, 25, 0.6), (9, 8, 14, 1.7),
                                             (32, 64, 46, None)])
def test_joseph_and_adjoint(N, na, nd, spacing):
    """The projector and its scattered adjoint equal the numpy oracle's (row and
    column walks, the 45-degree switch, bins wider and narrower than a pixel)."""
    g = operators.ParallelBeam(N, na, nd, 1.0 / N, (spacing or 1.0) / N)
    rng = np.random.default_rng(N + na)
    u, y = rng.random((N, N)), rng.standard_normal((na, nd))
    np.testing.assert_allclose(c.joseph(u, g), operators.joseph_forward(u, g), rtol=0, atol=1e-13)
    np.testing.assert_allclose(c.joseph(y, g, adjoint=True), operators.joseph_adjoint(y, g), rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", ["pgd", "fista", "proxskip"])
def test_ct_fb_solvers(kind):
    """PGD / FISTA / ProxSkip with the CT projector as A, as the numpy solvers run them."""
    N, na, nd = 20, 24, 29
    g = operators.ParallelBeam.unit_square(N, na, nd)
    rng = np.random.default_rng(3)
    b = operators.joseph_forward(rng.random((N, N)), g) + 0.01 * rng.standard_normal((na, nd))
    alpha, K, n_inner, p, seed = 0.002, 14, 6, 0.4, 11
    gamma = 0.9 / 1.6  # below 1 / ||A||^2 for this geometry (||A||^2 = 1.157 by the power method)
    prob = solvers.Problem(operators.ct_op(g), b, alpha, (N, N))
    x0 = np.zeros((N, N))
    if kind == "pgd":
        ref = solvers.pgd(prob, x0, gamma, K, n_inner)
    elif kind == "fista":
        ref = solvers.fista(prob, x0, gamma, K, n_inner)
    else:
        ref = solvers.proxskip(prob, x0, gamma, p, seed, K, n_inner)
    got = c.ct_fb_solve(kind, b, alpha, gamma, K, n_inner, g, p=p,
                        coins=coin.schedule(seed, p, K) if kind == "proxskip" else None)
    np.testing.assert_allclose(got["x"], ref["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["dual"], ref["dual"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(got["objective"], ref["objective"], rtol=1e-12)
    assert got["prox_calls"] == ref["prox_calls"] and got["iters_run"] == K


@pytest.mark.parametrize("nonneg", [False, True])
def test_ct_pdhg(nonneg):
    """Implicit PDHG with the CT projector, as the numpy solver runs it (K x-bar is
    formed from K x_{k+1} by linearity in C, directly in numpy)."""
    N, na, nd = 18, 22, 27
    g = operators.ParallelBeam.unit_square(N, na, nd)
    rng = np.random.default_rng(5)
    b = operators.joseph_forward(rng.random((N, N)), g) + 0.01 * rng.standard_normal((na, nd))
    alpha, K, n_inner, st = 0.003, 12, 7, 0.99 / np.sqrt(1.2)
    prob = solvers.Problem(operators.ct_op(g), b, alpha, (N, N), nonneg=nonneg)
    ref = solvers.pdhg(prob, np.zeros((N, N)), np.zeros((na, nd)), st, st, K, n_inner)
    got = c.ct_pdhg(b, alpha, st, st, K, n_inner, g, nonneg=nonneg)
    np.testing.assert_allclose(got["x"], ref["x"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got["y"], ref["y"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(got["objective"], ref["objective"], rtol=1e-12)


def test_joseph_full_size_adjoint():
    """At the CT workload's size (512^2, 720 x 725), the size of its F* run, the C
    projector and its adjoint pass the dot test <A u, y> = <u, A^T y>."""
    g = operators.ParallelBeam.unit_square(512, 720, 725)
    rng = np.random.default_rng(7)
    u, y = rng.random((512, 512)), rng.standard_normal((720, 725))
    au = c.joseph(u, g)
    lhs = float(np.sum(au * y))
    rhs = float(np.sum(u * c.joseph(y, g, adjoint=True)))
    # relative to the sum of the magnitudes of the terms (the sums cancel)
    assert abs(lhs - rhs) <= 1e-12 * float(np.abs(au * y).sum())
